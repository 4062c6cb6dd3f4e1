"""ctypes binding of the C ABI in include/es_vdw.h (argument marshalling only).

Every computation runs in ``libesvdw.so``; this module converts PyTorch CUDA
tensors to device pointers and Python settings to ``es_params``.  It raises if
the library is missing: there is no other code path.

Functions keep the C names: ``es_create``, ``es_init_mesh``, ``es_prim_to_cons``,
``es_rhs``, ``es_rk_stage``, ``es_cfl_dt``, ``es_mesh_redistribute``,
``es_step``, ``es_steps``, ``es_set_time``, ``es_get_time``, ``es_run_host``, ``es_check``.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libesvdw.so")

ES_OK, ES_ERR_ARG, ES_ERR_CUDA, ES_ERR_INADMISSIBLE, ES_ERR_MESH, ES_ERR_TIMEOUT = range(6)
ES_BC = {"periodic": 0, "outflow": 1, "reflect": 2, "symmetry_lo": 3}
ES_PREC = {"fp64": 0, "mixed": 1}
ES_MONITOR = {"vdw": 0, "smooth": 1}


class EsParams(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double), ("cv", ctypes.c_double),
        ("dim", ctypes.c_int), ("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
        ("dxi", ctypes.c_double * 3), ("period", ctypes.c_double * 3), ("bc", ctypes.c_int * 3),
        ("weno_gamma", ctypes.c_double * 3), ("weno_eps", ctypes.c_double), ("sign_tol", ctypes.c_double),
        ("dissipation", ctypes.c_int), ("cfl", ctypes.c_double), ("dt_fixed", ctypes.c_double),
        ("moving", ctypes.c_int), ("monitor", ctypes.c_int), ("kappa", ctypes.c_int),
        ("alpha", ctypes.c_double * 4), ("filter_passes", ctypes.c_int), ("jacobi_sweeps", ctypes.c_int),
        ("jacobi_eps", ctypes.c_double), ("precision", ctypes.c_int), ("tile", ctypes.c_int),
    ]


class EsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"es error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libesvdw.so (built by paper_2407_05568_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2407_05568_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.es_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(EsParams), vp]
        L.es_destroy.argtypes = [vp]
        L.es_destroy.restype = None
        L.es_init_mesh.argtypes = [vp, vp, vp]
        L.es_prim_to_cons.argtypes = [vp, vp, vp, vp, vp, vp]
        L.es_rhs.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.es_rk_stage.argtypes = [vp, i, d, vp, vp, vp, vp, vp, vp, vp, vp]
        L.es_cfl_dt.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(d)]
        L.es_mesh_redistribute.argtypes = [vp, vp, vp, vp, d, vp, ctypes.POINTER(i), ctypes.POINTER(d)]
        L.es_entropy_rate.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(d)]
        L.es_steps.argtypes = [vp, vp, vp, vp, i, d]
        L.es_step.argtypes = [vp, vp, vp, vp, d, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.es_set_time.argtypes = [vp, d]
        L.es_get_time.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.es_run_host.argtypes = [vp, vp, vp, vp, i, d]
        L.es_check.argtypes = [vp]
        L.es_last_error.argtypes = [vp, ctypes.c_char_p, i]
        L.es_autotune.argtypes = [vp, vp, vp, vp, ctypes.POINTER(i), ctypes.POINTER(d)]
        L.es_time_stage.argtypes = [vp, vp, vp, vp, i, d, i, ctypes.POINTER(d)]
        L.es_selftest_division.argtypes = [vp, vp, vp, vp, ctypes.c_int64, vp]
        L.es_selftest_division.restype = ctypes.c_int
        L.es_selftest_mixed_arith.argtypes = [vp, vp, vp, vp, ctypes.c_int64, vp, vp, vp, vp, vp]
        L.es_selftest_mixed_arith.restype = ctypes.c_int
        L.es_selftest_peaks.argtypes = [ctypes.POINTER(d), ctypes.POINTER(d), vp]
        L.es_selftest_peaks.restype = ctypes.c_int
        L.es_autotune.restype = ctypes.c_int
        L.es_launch_count.argtypes = [vp]
        L.es_launch_count.restype = ctypes.c_int64
        L.es_rk3_step_static.argtypes = [ctypes.POINTER(EsParams), d, vp, vp, vp, vp, vp]
        L.es_rk3_step_static.restype = ctypes.c_int
        L.es_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(EsParams), i, ctypes.POINTER(i), vp]
        L.es_batch_destroy.argtypes = [vp]
        L.es_batch_destroy.restype = None
        L.es_batch_nodes.argtypes = [vp]
        L.es_batch_nodes.restype = ctypes.c_int64
        L.es_batch_set_prim.argtypes = [vp, vp, vp, vp]
        L.es_batch_set_state.argtypes = [vp, vp, vp, vp, vp]
        L.es_batch_steps.argtypes = [vp, i, d]
        L.es_batch_autotune.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(d)]
        L.es_batch_get.argtypes = [vp, vp, vp, vp, vp]
        L.es_batch_check.argtypes = [vp]
        L.es_batch_last_error.argtypes = [vp, ctypes.c_char_p, i]
        L.es_mesh_features.argtypes = [vp, vp, vp, vp, vp]
        L.es_mesh_solve.argtypes = [vp, vp, vp, vp, vp, d, vp, vp, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.es_set_warm_start.argtypes = [vp, vp, vp, i, i, d]
        L.es_mesh_warm_start.argtypes = [vp, vp, vp, vp]
        L.es_mesh_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int64), i]
        L.es_nn_workspace_bytes.argtypes = [i, i, i, i, i]
        L.es_nn_workspace_bytes.restype = ctypes.c_size_t
        L.es_nn_conv_forward.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, vp, ctypes.c_size_t, vp]
        L.es_nn_conv_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, i, i, i, i, i, i, vp, ctypes.c_size_t, vp]
        L.es_nn_mse.argtypes = [vp, vp, vp, vp, ctypes.c_int64, vp]
        L.es_nn_conv_forward_bf16.argtypes = [vp, vp, vp, vp, i, i, i, i, i, i, vp]
        L.es_nn_to_bf16.argtypes = [vp, vp, ctypes.c_int64, vp]
        f = ctypes.c_float
        L.es_nn_adam.argtypes = [vp, vp, vp, vp, vp, i, f, f, f, f, i, vp]
        for name in ("es_mesh_features", "es_mesh_solve", "es_set_warm_start", "es_mesh_stats", "es_mesh_warm_start",
                     "es_nn_conv_forward", "es_nn_conv_backward", "es_nn_mse", "es_nn_adam", "es_nn_to_bf16",
                     "es_nn_conv_forward_bf16"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("es_batch_create", "es_batch_set_prim", "es_batch_set_state", "es_batch_steps", "es_batch_get", "es_batch_check",
                     "es_batch_autotune",
                     "es_batch_last_error"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("es_create", "es_init_mesh", "es_prim_to_cons", "es_rhs", "es_rk_stage", "es_cfl_dt",
                     "es_entropy_rate", "es_mesh_redistribute", "es_steps", "es_step", "es_set_time", "es_get_time", "es_run_host",
                     "es_check", "es_last_error"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def make_params(w, precision="fp64", dissipation=True, dt_fixed=0.0, weno_eps=1e-6, sign_tol=None, tile=0):
    """es_params from a workload description (see workloads.py)."""
    p = EsParams()
    g = w["gas"]
    p.a, p.b, p.R, p.cv = g["a"], g["b"], g["R"], g["cv"]
    p.dim = w["dim"]
    n = tuple(w["n"])[::-1]                     # workloads list sizes slowest axis first
    p.n1 = n[0]
    p.n2 = n[1] if w["dim"] >= 2 else 1
    p.n3 = n[2] if w["dim"] == 3 else 1
    for k in range(w["dim"]):
        p.dxi[k] = w["dxi"][k]
        p.period[k] = w["period"][k]
        p.bc[k] = ES_BC[w["bc"][k]]
    p.weno_gamma[:] = tuple(w.get("weno_gammas", (0.005, 0.045, 0.95)))
    p.weno_eps = weno_eps
    # round-off size of a zero plain jump, relative to the terms forming it: FP64
    # rounding, or a few FP32 roundings (the acoustic jumps of an entropy wave cancel
    # to 1e-7 of their terms near smooth extrema, below what FP32 resolves)
    p.sign_tol = sign_tol if sign_tol is not None else (1e-12 if precision == "fp64" else 4e-7)
    p.dissipation = int(dissipation)
    p.cfl = w.get("cfl", 0.4)
    p.dt_fixed = dt_fixed
    p.moving = int(w.get("moving", False))
    m = w.get("mesh", {})
    p.monitor = ES_MONITOR[m.get("monitor", "vdw")]
    p.kappa = m.get("kappa", 2)
    al = list(m.get("alphas", (1200.0, 1200.0, 1200.0)))
    for k, a in enumerate(al[:4]):
        p.alpha[k] = a
    p.filter_passes = m.get("filter_passes", 5)
    p.jacobi_sweeps = m.get("sweeps", 5)
    p.jacobi_eps = m.get("eps", 0.0)
    p.precision = ES_PREC[precision]
    p.tile = int(tile)
    return p


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype.is_floating_point and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float tensor")
    if dtype is not None and str(t.dtype) != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """Owns an es_ctx*; destroyed with the object."""

    def __init__(self, params, stream=None):
        self.params = params
        self.state_dtype = "torch.float32" if params.precision == ES_PREC["mixed"] else "torch.float64"
        self._h = ctypes.c_void_p()
        rc = lib().es_create(ctypes.byref(self._h), ctypes.byref(params), _stream_handle(stream))
        if rc != ES_OK:
            raise EsError(rc, "es_create rejected the parameters" if rc == ES_ERR_ARG else "es_create failed")

    def _call(self, rc):
        if rc != ES_OK:
            buf = ctypes.create_string_buffer(256)
            lib().es_last_error(self._h, buf, 256)
            raise EsError(rc, buf.value.decode())

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.es_destroy(self._h)
            self._h = None

    @property
    def launches(self):
        return int(lib().es_launch_count(self._h))


def es_create(params, stream=None):
    return Context(params, stream)


def state_empty(ctx, shape, device):
    """An uninitialised state array of the context's precision: float64 of `shape`, or in
    the mixed form the (hi, lo) float32 planes of shape (2, *shape)."""
    import torch
    if ctx.state_dtype == "torch.float32":
        return torch.empty((2,) + tuple(shape), dtype=torch.float32, device=device)
    return torch.empty(tuple(shape), dtype=torch.float64, device=device)


F64 = "torch.float64"
F32 = "torch.float32"
BF16 = "torch.bfloat16"


def es_init_mesh(ctx, x, J):
    ctx._call(lib().es_init_mesh(ctx._h, _ptr(x, F64), _ptr(J, ctx.state_dtype)))


def es_prim_to_cons(ctx, rho, v, p, J, JU):
    S = ctx.state_dtype
    ctx._call(lib().es_prim_to_cons(ctx._h, _ptr(rho, F64), _ptr(v, F64), _ptr(p, F64), _ptr(J, S), _ptr(JU, S)))


def es_rhs(ctx, JU, J, x, xdot, dJU, dJ):
    S = ctx.state_dtype
    ctx._call(lib().es_rhs(ctx._h, _ptr(JU, S), _ptr(J, S), _ptr(x, F64), _ptr(xdot, F64), _ptr(dJU, S),
                           _ptr(dJ, S)))


def es_rk_stage(ctx, stage, dt, JUn, Jn, JUs, Js, xn, xdot, JU_out, J_out):
    S = ctx.state_dtype
    ctx._call(lib().es_rk_stage(ctx._h, stage, dt, _ptr(JUn, S), _ptr(Jn, S), _ptr(JUs, S), _ptr(Js, S),
                                _ptr(xn, F64), _ptr(xdot, F64), _ptr(JU_out, S), _ptr(J_out, S)))


def es_cfl_dt(ctx, JU, J, x, xdot=None):
    """eq. cfl's time step; xdot (the mesh velocity, or None for a mesh at rest) enters the spectral radius."""
    S = ctx.state_dtype
    dt = ctypes.c_double()
    ctx._call(lib().es_cfl_dt(ctx._h, _ptr(JU, S), _ptr(J, S), _ptr(x, F64), _ptr(xdot, F64), ctypes.byref(dt)))
    return dt.value


def es_entropy_rate(ctx, JU, J, dJU, dJ):
    """FP64 entropy production check: (rate, sum of the magnitudes of its terms) of the total entropy."""
    S = ctx.state_dtype
    out = (ctypes.c_double * 2)()
    ctx._call(lib().es_entropy_rate(ctx._h, _ptr(JU, S), _ptr(J, S), _ptr(dJU, S), _ptr(dJ, S), out))
    return out[0], out[1]


def es_mesh_redistribute(ctx, JU, J, xn, dt, xdot, stats=True):
    """Sec. 4's redistribution from xn; returns (sweeps, Delta_gamma), or (None, None) with stats=False, which
    leaves the call asynchronous on the context's stream."""
    S = ctx.state_dtype
    sw = ctypes.c_int()
    gam = ctypes.c_double()
    ctx._call(lib().es_mesh_redistribute(ctx._h, _ptr(JU, S), _ptr(J, S), _ptr(xn, F64), dt, _ptr(xdot, F64),
                                         ctypes.byref(sw) if stats else None, ctypes.byref(gam) if stats else None))
    return (sw.value, gam.value) if stats else (None, None)


def es_mesh_features(ctx, JU, J, x, feat):
    """Warm-start features [4][n2][n1] (float32) at the mesh x."""
    S = ctx.state_dtype
    ctx._call(lib().es_mesh_features(ctx._h, _ptr(JU, S), _ptr(J, S), _ptr(x, F64), _ptr(feat, F32)))


def es_mesh_solve(ctx, JU, J, xn, x_start, x_out, disp_out=None, guard_ratio=1.0):
    """Jacobi solve of the mesh equation from xn (x_start None) or guarded from x_start;
    writes x_out (float64) and/or disp_out (float32, cells); returns (sweeps, picked)."""
    S = ctx.state_dtype
    sw = ctypes.c_int()
    pk = ctypes.c_int()
    ctx._call(lib().es_mesh_solve(ctx._h, _ptr(JU, S), _ptr(J, S), _ptr(xn, F64), _ptr(x_start, F64),
                                  float(guard_ratio), _ptr(x_out, F64), _ptr(disp_out, F32), ctypes.byref(sw),
                                  ctypes.byref(pk)))
    return sw.value, pk.value


def es_mesh_warm_start(ctx, xn, out, x_start):
    """x_start = xn + dxi out (out in cells, float32 [2][n2][n1]); fixed nodes keep xn."""
    ctx._call(lib().es_mesh_warm_start(ctx._h, _ptr(xn, F64), _ptr(out, F32), _ptr(x_start, F64)))


def es_set_warm_start(ctx, w_bf16, bias, layers, hidden, guard_ratio=1.0):
    """Register (or with w_bf16 None remove) the warm-start network; the context copies it."""
    ctx._call(lib().es_set_warm_start(ctx._h, _ptr(w_bf16, BF16), _ptr(bias, F32), int(layers), int(hidden),
                                      float(guard_ratio)))


def es_mesh_stats(ctx, reset=False):
    """(sweeps_total, solves, warm_kept) since the last reset."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    ctx._call(lib().es_mesh_stats(ctx._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), int(reset)))
    return a.value, b.value, c.value


def _nn_rc(rc, what):
    if rc != ES_OK:
        raise EsError(rc, f"{what} failed")


def es_nn_workspace_bytes(B, Cin, Cout, H, W):
    return int(lib().es_nn_workspace_bytes(int(B), int(Cin), int(Cout), int(H), int(W)))


def es_nn_conv_forward(inp, w, bias, out, act_tanh, workspace, stream=None):
    """out = act(bias + w (*) inp) for inp [B][Cin][H][W], w [Cout][Cin][3][3] bf16."""
    B, Cin, H, W = inp.shape
    Cout = w.shape[0]
    _nn_rc(lib().es_nn_conv_forward(_ptr(inp, F32), _ptr(w, BF16), _ptr(bias, F32), _ptr(out, F32), B, Cin, Cout,
                                    H, W, int(act_tanh), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                    _stream_handle(stream)), "es_nn_conv_forward")


def es_nn_conv_forward_bf16(inp, w, bias, out, act_tanh, stream=None):
    """The same layer on the tensor cores: input rounded to bf16, FP32 accumulation."""
    B, Cin, H, W = inp.shape
    Cout = w.shape[0]
    _nn_rc(lib().es_nn_conv_forward_bf16(_ptr(inp, F32), _ptr(w, BF16), _ptr(bias, F32), _ptr(out, F32), B, Cin,
                                         Cout, H, W, int(act_tanh), _stream_handle(stream)), "es_nn_conv_forward_bf16")


def es_nn_conv_backward(inp, w, out, grad_out, grad_in, grad_w, grad_b, act_tanh, workspace, stream=None):
    B, Cin, H, W = inp.shape
    Cout = w.shape[0]
    _nn_rc(lib().es_nn_conv_backward(_ptr(inp, F32), _ptr(w, BF16), _ptr(out, F32), _ptr(grad_out, F32),
                                     _ptr(grad_in, F32), _ptr(grad_w, F32), _ptr(grad_b, F32), B, Cin, Cout, H, W,
                                     int(act_tanh), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                     _stream_handle(stream)), "es_nn_conv_backward")


def es_nn_to_bf16(src, dst, stream=None):
    _nn_rc(lib().es_nn_to_bf16(_ptr(src, F32), _ptr(dst, BF16), src.numel(), _stream_handle(stream)),
           "es_nn_to_bf16")


def es_nn_mse(pred, target, grad, loss, stream=None):
    _nn_rc(lib().es_nn_mse(_ptr(pred, F32), _ptr(target, F32), _ptr(grad, F32), _ptr(loss, F32), pred.numel(),
                           _stream_handle(stream)), "es_nn_mse")


def es_nn_adam(master, w_bf16, grad, m, v, lr, beta1, beta2, eps, step, stream=None):
    _nn_rc(lib().es_nn_adam(_ptr(master, F32), _ptr(w_bf16, BF16), _ptr(grad, F32), _ptr(m, F32), _ptr(v, F32),
                            master.numel(), float(lr), float(beta1), float(beta2), float(eps), int(step),
                            _stream_handle(stream)), "es_nn_adam")


def es_steps(ctx, JU, J, x, nsteps, t_end):
    S = ctx.state_dtype
    ctx._call(lib().es_steps(ctx._h, _ptr(JU, S), _ptr(J, S), _ptr(x, F64), int(nsteps), float(t_end)))


def es_step(ctx, JU, J, x, t_end):
    """One full step; returns (time after the step, step taken)."""
    S = ctx.state_dtype
    t = ctypes.c_double()
    dt = ctypes.c_double()
    ctx._call(lib().es_step(ctx._h, _ptr(JU, S), _ptr(J, S), _ptr(x, F64), float(t_end), ctypes.byref(t),
                            ctypes.byref(dt)))
    return t.value, dt.value


def es_set_time(ctx, t):
    ctx._call(lib().es_set_time(ctx._h, float(t)))


def es_get_time(ctx):
    t = ctypes.c_double()
    dt = ctypes.c_double()
    ctx._call(lib().es_get_time(ctx._h, ctypes.byref(t), ctypes.byref(dt)))
    return t.value, dt.value


def es_run_host(ctx, JU, J, x, nsteps, t_end):
    """JU, J (state precision) and x (float64): C-contiguous numpy arrays in host memory, updated in place."""
    arrs = [JU, J, x]
    sdt = np.float32 if ctx.state_dtype == "torch.float32" else np.float64
    for a, dt in zip(arrs, (sdt, sdt, np.float64)):
        if not (isinstance(a, np.ndarray) and a.dtype == dt and a.flags.c_contiguous):
            raise ValueError("expected C-contiguous arrays of the state precision (x: float64)")
    ptrs = [ctypes.c_void_p(a.ctypes.data) for a in arrs]
    ctx._call(lib().es_run_host(ctx._h, *ptrs, int(nsteps), float(t_end)))


def es_autotune(ctx, JU, J, x):
    """Time the stage kernel's tile shapes on this state; returns (chosen shape 1..5, [ms per shape])."""
    S = ctx.state_dtype
    k = ctypes.c_int()
    ms = (ctypes.c_double * 5)()
    ctx._call(lib().es_autotune(ctx._h, _ptr(JU, S), _ptr(J, S), _ptr(x, F64), ctypes.byref(k), ms))
    return k.value, list(ms)


def es_time_stage(ctx, JU, J, x, stage=2, dt=1e-4, reps=20):
    """Mean device time (ms) of `reps` back-to-back launches of the fused stage kernel (1D/2D)."""
    S = ctx.state_dtype
    ms = ctypes.c_double()
    ctx._call(lib().es_time_stage(ctx._h, _ptr(JU, S), _ptr(J, S), _ptr(x, F64), int(stage), float(dt), int(reps),
                                  ctypes.byref(ms)))
    return ms.value


def es_selftest_division(a, b, q, r, stream=None):
    """q = a / b and r = 1 / b with the library's FP64 division (float64 device arrays)."""
    _nn_rc(lib().es_selftest_division(_ptr(a, F64), _ptr(b, F64), _ptr(q, F64), _ptr(r, F64), a.numel(),
                                      _stream_handle(stream)), "es_selftest_division")


def es_selftest_mixed_arith(x, f, a, b, stream=None):
    """Device self-test of the mixed form's building blocks (see es_vdw.h): x (float64, n), f (float32, n),
    a and b (float32, 2n: double-float pairs).  Returns (split, wide, mul, add) as device tensors."""
    import torch
    n = x.numel()
    split = torch.empty(2 * n, dtype=torch.float32, device=x.device)
    wide = torch.empty(n, dtype=torch.float64, device=x.device)
    mul = torch.empty(2 * n, dtype=torch.float32, device=x.device)
    add = torch.empty(2 * n, dtype=torch.float32, device=x.device)
    _nn_rc(lib().es_selftest_mixed_arith(_ptr(x, F64), _ptr(f, F32), _ptr(a, F32), _ptr(b, F32), n, _ptr(split, F32),
                                         _ptr(wide, F64), _ptr(mul, F32), _ptr(add, F32), _stream_handle(stream)),
           "es_selftest_mixed_arith")
    return split, wide, mul, add


def es_selftest_peaks(stream=None):
    """Measured (FP64, FP32) FMA-chain rates of the current GPU in TFLOP/s."""
    f64, f32 = ctypes.c_double(), ctypes.c_double()
    rc = lib().es_selftest_peaks(ctypes.byref(f64), ctypes.byref(f32), _stream_handle(stream))
    if rc != ES_OK:
        raise EsError(rc, "es_selftest_peaks failed")
    return f64.value, f32.value


def es_check(ctx):
    """Synchronise and return the latched device status (0 = ok)."""
    return int(lib().es_check(ctx._h))


def es_rk3_step_static(params, dt, JU, J, x, xdot=None, stream=None):
    """Allocation-free SSP-RK3 step (see es_vdw.h); returns the status code (0 = ok)."""
    return int(lib().es_rk3_step_static(ctypes.byref(params), float(dt), _ptr(JU), _ptr(J), _ptr(x),
                                        _ptr(xdot), _stream_handle(stream)))


class Batch:
    """Owns an es_batch* (many 1D problems advanced by one persistent launch)."""

    def __init__(self, params, lengths, stream=None):
        self.lengths = np.ascontiguousarray(np.asarray(lengths, dtype=np.int32))
        self.nprob = int(self.lengths.size)
        self._h = ctypes.c_void_p()
        arr = self.lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        rc = lib().es_batch_create(ctypes.byref(self._h), ctypes.byref(params), self.nprob, arr,
                                   _stream_handle(stream))
        if rc != ES_OK:
            raise EsError(rc, "es_batch_create rejected the parameters")
        self.ntot = int(lib().es_batch_nodes(self._h))
        self.offsets = np.concatenate([[0], np.cumsum(self.lengths)[:-1]]).astype(np.int64)

    def _call(self, rc):
        if rc != ES_OK:
            buf = ctypes.create_string_buffer(256)
            lib().es_batch_last_error(self._h, buf, 256)
            raise EsError(rc, buf.value.decode())

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.es_batch_destroy(self._h)
            self._h = None


def es_batch_create(params, lengths, stream=None):
    return Batch(params, lengths, stream)


def es_batch_set_prim(b, rho, v, p):
    b._call(lib().es_batch_set_prim(b._h, _ptr(rho, F64), _ptr(v, F64), _ptr(p, F64)))


def es_batch_set_state(b, JU, J, x, t):
    """Every problem's conservative state, mesh and time (device float64 arrays, es_batch_get's layout)."""
    b._call(lib().es_batch_set_state(b._h, _ptr(JU, F64), _ptr(J, F64), _ptr(x, F64), _ptr(t, F64)))


def es_batch_steps(b, nsteps, t_end):
    b._call(lib().es_batch_steps(b._h, int(nsteps), float(t_end)))


def es_batch_autotune(b):
    """Time one step of each CTA shape from the current state (restored afterwards) and keep
    the fastest; returns (threads per CTA, [probe ms for 128, 256, 512])."""
    bt = ctypes.c_int()
    ms = (ctypes.c_double * 3)()
    b._call(lib().es_batch_autotune(b._h, ctypes.byref(bt), ms))
    return bt.value, list(ms)


def es_batch_get(b, JU, J, x, t=None):
    b._call(lib().es_batch_get(b._h, _ptr(JU, F64), _ptr(J, F64), _ptr(x, F64), _ptr(t, F64)))


def es_batch_check(b):
    return int(lib().es_batch_check(b._h))


def batch_params(gas, cfl=0.4, alphas=(1200.0, 1200.0, 1200.0), kappa=2, filter_passes=5, sweeps=5,
                 moving=True, sign_tol=4e-7):
    """es_params for es_batch_create: 1D, mixed form, vdW monitor (Sec. 4)."""
    w = dict(gas=gas, dim=1, n=(8,), dxi=(1.0,), bc=("outflow",), period=(1.0,), cfl=cfl, moving=moving,
             mesh=dict(monitor="vdw", alphas=alphas, kappa=kappa, filter_passes=filter_passes, sweeps=sweeps))
    return make_params(w, precision="mixed", sign_tol=sign_tol)


def es_last_error(ctx):
    buf = ctypes.create_string_buffer(256)
    lib().es_last_error(ctx._h, buf, 256)
    return buf.value.decode()


def setup_workload(w, precision="fp64", device="cuda", dissipation=True, dt_fixed=0.0, stream=None):
    """Context and device state (JU, J, x) of a workload description (workloads.py): J from
    the mesh, JU from the primitive fields, time 0.  dt_fixed > 0 replaces the CFL step.
    `stream` (a torch.cuda.Stream, or None for the current one) carries the context's work."""
    import contextlib

    import torch
    dev = torch.device(device)
    ctx = es_create(make_params(w, precision=precision, dissipation=dissipation, dt_fixed=dt_fixed), stream)
    with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
        x = torch.tensor(np.ascontiguousarray(w["x"]), dtype=torch.float64, device=dev)
        J = state_empty(ctx, w["x"].shape[1:], dev)
        es_init_mesh(ctx, x, J)
        rho = torch.tensor(w["rho"], dtype=torch.float64, device=dev)
        v = torch.tensor(np.ascontiguousarray(w["v"]), dtype=torch.float64, device=dev)
        p = torch.tensor(w["p"], dtype=torch.float64, device=dev)
        JU = state_empty(ctx, (w["dim"] + 2,) + w["x"].shape[1:], dev)
        es_prim_to_cons(ctx, rho, v, p, J, JU)
    if stream is not None:
        stream.synchronize()
    es_set_time(ctx, 0.0)
    return ctx, JU, J, x
