"""The mixed-precision form (stage arithmetic on the FP32 pipe) against the FP64 oracle.

Bar: <= 1e-5 relative L1 against the oracle at the final time on smooth
problems, with the design order of the scheme preserved above the FP32 floor.
The operator itself agrees to 2e-6 of the flux scale sum|JU|/dxi (1e-6 for the
EC part alone).  On discontinuous data the sign switch Y takes some decisions
differently in FP32 (a plain jump within a few FP32 roundings of its terms
counts as zero), so the bound there is 1e-4 after a few steps.
"""
import numpy as np
import pytest

from oracle import operator as op
from oracle import stepper
from paper_2407_05568_gb300 import workloads as wl

from sides import gpu_setup, oracle_setup, rel_l1, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_05568_gb300 import build
    build.build()


def _wavy(n=40):
    w = wl.sine_2d(n)
    X, Y = w["x"]
    w["x"] = wl.wavy_mesh_2d(X, Y)
    w["rho"], w["v"], w["p"] = wl.smooth_state_2d(X, Y)
    w["xdot"] = wl.mesh_velocity_2d(X, Y)
    return w


@pytest.mark.parametrize("dissipation", [False, True])
@pytest.mark.parametrize("case", ["sine1d", "sine2d", "wavy", "vortex"])
def test_mixed_rhs_vs_oracle(case, dissipation):
    import torch

    from paper_2407_05568_gb300 import es
    w = {"sine1d": lambda: wl.sine_1d(200), "sine2d": lambda: wl.sine_2d(96), "wavy": lambda: _wavy(64),
         "vortex": lambda: wl.isentropic_vortex(64)}[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w, dissipation=dissipation)
    ctx, JU, J, xt = gpu_setup(w, precision="mixed", dissipation=dissipation)
    xd = w.get("xdot", np.zeros_like(w["x"]))
    dU_o, dJ_o = op.rhs(sch, JU_o, J_o, x, xd)
    xdt = torch.tensor(np.ascontiguousarray(xd), dtype=torch.float64, device="cuda")
    dU = torch.empty_like(JU)
    dJ = torch.empty_like(J)
    es.es_rhs(ctx, JU, J, xt, xdt, dU, dJ)
    assert es.es_check(ctx) == 0
    scale = np.abs(JU_o).sum() / min(w["dxi"])
    err = np.abs(to_np(dU) - dU_o).sum() / scale
    assert err < (2e-6 if dissipation else 1e-6), err


def _run_both(w, t_end, dt_fixed=None):
    from paper_2407_05568_gb300 import es
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    JU_o, J_o, x_o, n = stepper.run(sch, mc, JU_o, J_o, x_o, t_end, w["cfl"], dt_fixed=dt_fixed)
    ctx, JU, J, xt = gpu_setup(w, precision="mixed", dt_fixed=dt_fixed or 0.0)
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, n + 2, t_end)
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    t, _ = es.es_get_time(ctx)
    assert t == pytest.approx(t_end, rel=1e-12)
    return JU_o, J_o, x_o, to_np(JU), to_np(J), to_np(xt)


@pytest.mark.parametrize("case", ["sine1d", "sine2d", "vortex"])
def test_mixed_final_time_vs_oracle(case):
    """Relative L1 of (JU, J) against the FP64 oracle at the final time <= 1e-5."""
    w, t_end = {"sine1d": (wl.sine_1d(200), 0.1), "sine2d": (wl.sine_2d(96), 0.05),
                "vortex": (wl.isentropic_vortex(64), 0.5)}[case]
    JU_o, J_o, x_o, JU, J, x = _run_both(w, t_end)
    assert rel_l1(JU, JU_o) < 1e-5, rel_l1(JU, JU_o)
    assert rel_l1(J, J_o) < 1e-6


def test_mixed_riemann_moving_mesh_few_steps():
    """The 2D vdW Riemann problem on the moving mesh, 3 steps (discontinuous data)."""
    w = wl.riemann_2d(64, seed=5)
    from paper_2407_05568_gb300 import es
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    t = 0.0
    for _ in range(3):
        JU_o, J_o, x_o, t, _ = stepper.step(sch, mc, JU_o, J_o, x_o, t, w["t_end"], w["cfl"])
    ctx, JU, J, xt = gpu_setup(w, precision="mixed")
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, 3, w["t_end"])
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    assert rel_l1(to_np(JU), JU_o) < 1e-4, rel_l1(to_np(JU), JU_o)
    assert rel_l1(to_np(xt), x_o) < 1e-5


def test_mixed_design_order_1d():
    """Example 5.1 setup (fixed mesh, dt = 0.4 dxi^(5/3)): the mixed form keeps ~5th order."""
    from paper_2407_05568_gb300 import es
    errs = []
    for n in (20, 40, 80):
        w = wl.sine_1d(n, t_end=0.05)
        dt = 0.4 * w["dxi"][0] ** (5.0 / 3.0)
        ctx, JU, J, xt = gpu_setup(w, precision="mixed", dt_fixed=dt)
        es.es_set_time(ctx, 0.0)
        es.es_steps(ctx, JU, J, xt, int(np.ceil(w["t_end"] / dt)) + 2, w["t_end"])
        assert es.es_check(ctx) == 0
        rho = to_np(JU)[0] / to_np(J)
        ex = 0.5 + 0.2 * np.sin(2 * np.pi * (w["x"][0] - w["t_end"]))
        errs.append(np.abs(rho - ex).mean())
    order = np.log2(errs[-2] / errs[-1])
    assert order > 4.5, errs


@pytest.mark.parametrize("case", ["riemann2d", "rp1d", "wavy_periodic", "riemann2d_mm1"])
def test_mixed_mesh_redistribution_fp32_vs_oracle(case):
    """The mixed form's time step and mesh redistribution run on the FP32 displacement:
    the same sweeps, Delta_gamma and mesh velocity as the FP64 oracle to FP32 rounding."""
    import torch

    from paper_2407_05568_gb300 import es
    if case == "riemann2d":
        w = wl.riemann_2d(64, seed=5)
    elif case == "riemann2d_mm1":                  # monitor without G (MM1)
        w = wl.mm1(wl.riemann_2d(64, seed=5))
    elif case == "rp1d":
        w = wl.riemann_1d("RP1", n=300)
    else:
        w = _wavy(48)
        w["moving"] = True
        w["mesh"] = dict(monitor="vdw", alphas=(1200.0, 1200.0, 1200.0), kappa=2, filter_passes=5, sweeps=5,
                         eps=0.0)
        w["rho"], w["v"], w["p"] = wl.rough_state(w["x"].shape[1:], 11, 2)
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w, precision="mixed")
    dt = 0.004
    xdot_o, sw_o, gam_o = stepper.redistribute(sch, mc, JU_o, J_o, x, dt)
    xdot = torch.empty_like(xt)
    sw, gam = es.es_mesh_redistribute(ctx, JU, J, xt, dt, xdot)
    assert sw == sw_o
    assert abs(gam - gam_o) <= 1e-5 * gam_o
    assert np.abs(to_np(xdot) - xdot_o).max() <= 2e-5 * np.abs(xdot_o).max()
    dt_o = stepper.cfl_dt(sch, JU_o, J_o, x, w.get("cfl", 0.4))
    assert abs(es.es_cfl_dt(ctx, JU, J, xt) - dt_o) <= 1e-5 * dt_o


@pytest.mark.parametrize("case", ["riemann2d", "wavy_periodic"])
def test_mixed_fused_sweeps_match_per_sweep_kernels(case):
    """The fused multi-sweep Jacobi kernel (no tolerance) and the per-sweep kernels (forced by a
    tolerance that is never met) give the same mesh velocity to FP32 rounding."""
    import torch

    from paper_2407_05568_gb300 import es
    w = wl.riemann_2d(70, seed=5) if case == "riemann2d" else _wavy(48)
    if case == "wavy_periodic":
        w["moving"] = True
        w["mesh"] = dict(monitor="vdw", alphas=(1200.0, 1200.0, 1200.0), kappa=2, filter_passes=5, sweeps=5,
                         eps=0.0)
        w["rho"], w["v"], w["p"] = wl.rough_state(w["x"].shape[1:], 11, 2)
    out = []
    for eps in (0.0, 1e-300):
        w["mesh"] = dict(w["mesh"], sweeps=6, eps=eps)
        ctx, JU, J, xt = gpu_setup(w, precision="mixed")
        xdot = torch.empty_like(xt)
        sw, gam = es.es_mesh_redistribute(ctx, JU, J, xt, 0.004, xdot)
        assert sw == 6
        out.append((to_np(xdot), gam))
    scale = np.abs(out[1][0]).max()
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-6 * scale
    assert abs(out[0][1] - out[1][1]) <= 1e-6 * out[1][1]


def test_mixed_free_stream_on_a_moving_mesh():
    """A constant state on the moving wavy periodic mesh (Remark after eq. HOstable) in the mixed form: the metrics
    come from the FP32 displacement, so the discrete SCL holds to FP32 rounding of the metric differences rather
    than exactly; over 5 full RK steps (15 stages) the state moves by a few FP32 roundings of its size: 3.3e-7
    measured, bar 1e-6 (the FP64 form: 1e-12)."""
    import torch

    from paper_2407_05568_gb300 import es
    w = _wavy(32)
    X = w["x"][0]
    w["rho"] = np.full_like(X, 0.8)
    w["v"] = np.stack([np.full_like(X, 0.3), np.full_like(X, -0.2)])
    w["p"] = np.full_like(X, 1.1)
    ctx, JU, J, xt = gpu_setup(w, precision="mixed")
    U0 = to_np(JU) / to_np(J)
    xdt = torch.tensor(w["xdot"], dtype=torch.float64, device="cuda")
    dt = 0.2 * w["dxi"][0]
    a = (torch.empty_like(JU), torch.empty_like(J))
    b = (torch.empty_like(JU), torch.empty_like(J))
    for _ in range(5):
        es.es_rk_stage(ctx, 1, dt, JU, J, JU, J, xt, xdt, *a)
        es.es_rk_stage(ctx, 2, dt, JU, J, a[0], a[1], xt, xdt, *b)
        es.es_rk_stage(ctx, 3, dt, JU, J, b[0], b[1], xt, xdt, JU, J)
        xt += dt * xdt
    assert es.es_check(ctx) == 0
    dev = np.abs(to_np(JU) / to_np(J) - U0).max() / np.abs(U0).max()
    assert dev < 1e-6, dev


def test_mixed_riemann_2d_every_step():
    """The 2D moving-mesh vdW Riemann problem (64^2, seed 5): over its first 40 steps, each mixed-form step taken
    from the oracle's state equals the oracle's next state within 1e-5 relative L1 (JU, J, x); the double-float
    monitor G keeps the mesh velocity at the oracle's near the critical point."""
    import torch

    from paper_2407_05568_gb300 import es
    w = wl.riemann_2d(64, seed=5)
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w, precision="mixed")
    t = 0.0
    worst = 0.0
    for k in range(40):
        for arr, dst in ((JU_o, JU), (J_o, J)):
            hi = arr.astype(np.float32)
            dst[0].copy_(torch.from_numpy(hi))
            dst[1].copy_(torch.from_numpy((arr - hi.astype(np.float64)).astype(np.float32)))
        xt.copy_(torch.from_numpy(x_o))
        es.es_set_time(ctx, t)
        es.es_steps(ctx, JU, J, xt, 1, w["t_end"])
        JU_o, J_o, x_o, t, _ = stepper.step(sch, mc, JU_o, J_o, x_o, t, w["t_end"], w["cfl"])
        err = max(rel_l1(to_np(JU), JU_o), rel_l1(to_np(J), J_o), rel_l1(to_np(xt), x_o))
        worst = max(worst, err)
        assert err < 1e-5, (k, err)
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    assert worst > 0.0


def test_mixed_arith_building_blocks():
    """The bit-level float <-> double moves of the mixed form's elementwise kernels and its double-float
    product and sum, against exact arithmetic (fractions): the split of a double is within 2^-46 of it
    (relative) with hi its truncation; widening is exact for every float class (zeros, subnormals,
    infinities, quiet NaNs with payload); the double-float product is within 2^-44 of the exact product of
    its inputs, the sum within 2^-44 of |a| + |b| (the sum's bound allows cancellation)."""
    from fractions import Fraction

    import torch

    from paper_2407_05568_gb300 import es
    rng = np.random.default_rng(7)
    n = 3000
    x = rng.standard_normal(n) * 10.0 ** rng.uniform(-30, 30, n)
    x[:12] = [0.0, -0.0, 1.0, -1.5, 2.0 ** -103, -(2.0 ** -103), 2.0 ** 127 * 1.999, 1e-200, 1e-310, 3.0, 0.1, 1e3]
    f = (rng.standard_normal(n) * 10.0 ** rng.uniform(-30, 30, n)).astype(np.float32)
    special = np.array([0x00000001, 0x80000003, 0x007fffff, 0x00400000, 0x80000000, 0x00000000, 0x7f800000,
                        0xff800000, 0x7fc00000, 0x7fc01234, 0x3f800000, 0x00012345], dtype=np.uint32)
    f[:special.size] = special.view(np.float32)
    hi = rng.uniform(-2, 2, (2, n)) * 10.0 ** rng.uniform(-3, 3, (2, n))
    pairs = []
    for h in hi:
        h32 = h.astype(np.float32)
        lo32 = (h32.astype(np.float64) * rng.uniform(-1, 1, n) * 2.0 ** -24).astype(np.float32)
        pairs.append(np.stack([h32, lo32], axis=1).reshape(-1))
    dev = lambda v: torch.tensor(v, device="cuda")
    split, wide, mul, add = es.es_selftest_mixed_arith(dev(x), dev(f), dev(pairs[0]), dev(pairs[1]))
    torch.cuda.synchronize()
    split, wide, mul, add = (t.cpu().numpy() for t in (split, wide, mul, add))
    sh, sl = split[0::2].astype(np.float64), split[1::2].astype(np.float64)
    ax = np.abs(x)
    inr = (ax >= 2.0 ** -103) & (ax < 2.0 ** 128)
    assert inr.sum() > n // 2
    assert np.all(np.abs(x[inr] - (sh[inr] + sl[inr])) <= 2.0 ** -46 * ax[inr])
    assert np.all(np.abs(sh[inr]) <= ax[inr]) and np.all(np.sign(sh[inr]) == np.sign(x[inr]))
    assert np.all(ax[inr] - np.abs(sh[inr]) < np.spacing(np.abs(split[0::2][inr])).astype(np.float64))
    assert sh[0] == 0.0 and sl[0] == 0.0 and sh[1] == 0.0
    ref = f.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(wide[~nan].view(np.uint64), ref[~nan].view(np.uint64))
    assert np.array_equal(wide[nan].view(np.uint64), ref[nan].view(np.uint64))   # quiet NaNs: payload kept
    worst_mul = worst_add = 0.0
    for i in range(n):
        A = Fraction(float(pairs[0][2 * i])) + Fraction(float(pairs[0][2 * i + 1]))
        B = Fraction(float(pairs[1][2 * i])) + Fraction(float(pairs[1][2 * i + 1]))
        P = Fraction(float(mul[2 * i])) + Fraction(float(mul[2 * i + 1]))
        S = Fraction(float(add[2 * i])) + Fraction(float(add[2 * i + 1]))
        worst_mul = max(worst_mul, float(abs(P - A * B) / abs(A * B)))
        worst_add = max(worst_add, float(abs(S - (A + B)) / (abs(A) + abs(B))))
    assert worst_mul <= 2.0 ** -44, worst_mul
    assert worst_add <= 2.0 ** -44, worst_add


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_steps_in_one_call_match_single_steps(precision):
    """es_steps(K) replays a first-step graph and then a continuation graph whose advance kernel formed the next
    step's FP32 displacement and reset the reductions (no displacement or reset kernel at its start); on the
    Riemann problem (outflow ends: the displacement's origin node does not move) it gives the same state, mesh
    and time bit for bit as K calls of one step."""
    import torch

    from paper_2407_05568_gb300 import es
    w = wl.riemann_2d(48, seed=5)
    out = []
    for mode in ("one_call", "single_steps"):
        ctx, JU, J, xt = gpu_setup(w, precision=precision)
        if mode == "one_call":
            es.es_steps(ctx, JU, J, xt, 4, w["t_end"])
        else:
            for _ in range(4):
                es.es_steps(ctx, JU, J, xt, 1, w["t_end"])
        torch.cuda.synchronize()
        assert es.es_check(ctx) == 0, es.es_last_error(ctx)
        out.append((to_np(JU), to_np(J), to_np(xt), es.es_get_time(ctx)))
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
    assert out[0][3] == out[1][3]


@pytest.mark.parametrize("passes,sweeps", [(1, 1), (8, 8), (3, 2)])
@pytest.mark.parametrize("case", ["riemann2d", "wavy_periodic"])
def test_mixed_register_tiles_vs_oracle(case, passes, sweeps):
    """The register-tiled filter and sweep kernels at the ends of their halo range (1 and 8 passes or sweeps: tiles
    with 62 and 48 output columns) on outflow and periodic meshes whose sizes leave ragged tiles: the same sweeps,
    Delta_gamma and mesh velocity as the FP64 oracle to FP32 rounding."""
    import torch

    from paper_2407_05568_gb300 import es
    if case == "riemann2d":
        w = wl.riemann_2d(70, seed=5)
    else:
        w = _wavy(52)
        w["moving"] = True
        w["rho"], w["v"], w["p"] = wl.rough_state(w["x"].shape[1:], 11, 2)
    w["mesh"] = dict(monitor="vdw", alphas=(1200.0, 1200.0, 1200.0), kappa=2, filter_passes=passes, sweeps=sweeps,
                     eps=0.0)
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w, precision="mixed")
    dt = 0.004
    xdot_o, sw_o, gam_o = stepper.redistribute(sch, mc, JU_o, J_o, x, dt)
    xdot = torch.empty_like(xt)
    sw, gam = es.es_mesh_redistribute(ctx, JU, J, xt, dt, xdot)
    assert sw == sw_o == sweeps
    assert abs(gam - gam_o) <= 1e-5 * gam_o
    assert np.abs(to_np(xdot) - xdot_o).max() <= 2e-5 * np.abs(xdot_o).max()
