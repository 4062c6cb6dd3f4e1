"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bar (FP64 form): one full time step agrees with the oracle to <= 1e-12 relative
L1 in (JU, J, x).  The bare operator is a difference quotient of O(1) fluxes,
so its parity is stated relative to the flux scale sum|JU|/dxi (also 1e-12).
Sizes span several CTA tiles (32 x 8 in 2D, 256 in 1D) and ragged tails.
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


def _ragged_riemann(n1=70, n2=45, seed=3):
    w = wl.riemann_2d(8, seed=seed)
    x1, d1 = wl.uniform_nodes(n1, 0.0, 1.0, False)
    x2, d2 = wl.uniform_nodes(n2, 0.0, 1.0, False)
    X, Y = np.meshgrid(x1, x2)
    st = np.array(wl.quadrant_states(seed))
    q = np.where(X > 0.5, np.where(Y > 0.5, 0, 3), np.where(Y > 0.5, 1, 2))
    w.update(n=(n2, n1), dxi=(d1, d2), x=np.stack([X, Y]), rho=st[q, 0], v=np.stack([st[q, 1], st[q, 2]]),
             p=st[q, 3])
    return w


def _wavy_periodic(n=40, rough=False):
    w = wl.sine_2d(n)
    X, Y = w["x"]
    w["x"] = wl.wavy_mesh_2d(X, Y)
    if rough:
        w["rho"], w["v"], w["p"] = wl.rough_state(X.shape, 11, 2)
    else:
        w["rho"], w["v"], w["p"] = wl.smooth_state_2d(X, Y)
    w["xdot"] = wl.mesh_velocity_2d(X, Y)
    return w


def _rp1d(n=300):
    return wl.riemann_1d("RP1", n=n)


CASES = {
    "sine1d": lambda: wl.sine_1d(200),
    "rp1d_ragged": lambda: _rp1d(300),
    "riemann2d_ragged": _ragged_riemann,
    "wavy_periodic": _wavy_periodic,
    "wavy_rough": lambda: _wavy_periodic(36, rough=True),
    "vortex_ideal": lambda: wl.isentropic_vortex(48),
}


def _xdot(w):
    if "xdot" in w:
        return w["xdot"]
    return np.zeros_like(w["x"])


@pytest.mark.parametrize("case", list(CASES))
def test_init_parity(case):
    w = CASES[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    assert rel_l1(to_np(J), J_o) < 1e-14
    assert rel_l1(to_np(JU), JU_o) < 1e-14


@pytest.mark.parametrize("dissipation", [True, False])
@pytest.mark.parametrize("case", list(CASES))
def test_rhs_parity(case, dissipation):
    import torch

    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w, dissipation=dissipation)
    ctx, JU, J, xt = gpu_setup(w, dissipation=dissipation)
    xd = _xdot(w)
    dU_o, dJ_o = op.rhs(sch, JU_o, J_o, x, xd)
    xdt = torch.tensor(np.ascontiguousarray(xd), dtype=torch.float64, device="cuda")
    dU = torch.empty_like(JU)
    dJ = torch.empty_like(J)
    es.es_rhs(ctx, JU, J, xt, xdt, dU, dJ)
    assert es.es_check(ctx) == 0
    scale = np.abs(JU_o).sum() / min(w["dxi"])
    err = np.abs(to_np(dU) - dU_o).sum() / scale
    assert err < 1e-12, err
    errJ = np.abs(to_np(dJ) - dJ_o).sum() / (np.abs(J_o).sum() / min(w["dxi"]))
    assert errJ < 1e-12, errJ
    # and the operator itself is not trivially zero
    assert np.abs(dU_o).sum() > 1e-6 * scale * min(w["dxi"])


@pytest.mark.parametrize("case", ["sine1d", "riemann2d_ragged", "wavy_periodic"])
def test_rk_stage_parity(case):
    import torch

    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    xd = _xdot(w)
    xdt = torch.tensor(np.ascontiguousarray(xd), dtype=torch.float64, device="cuda")
    dt = 0.3 * min(w["dxi"])
    o1 = stepper.rk_stage(sch, 0, dt, JU_o, J_o, JU_o, J_o, x, xd)
    o2 = stepper.rk_stage(sch, 1, dt, JU_o, J_o, o1[0], o1[1], x, xd)
    o3 = stepper.rk_stage(sch, 2, dt, JU_o, J_o, o2[0], o2[1], x, xd)
    g1 = (torch.empty_like(JU), torch.empty_like(J))
    g2 = (torch.empty_like(JU), torch.empty_like(J))
    g3 = (torch.empty_like(JU), torch.empty_like(J))
    es.es_rk_stage(ctx, 1, dt, JU, J, JU, J, xt, xdt, *g1)
    es.es_rk_stage(ctx, 2, dt, JU, J, g1[0], g1[1], xt, xdt, *g2)
    es.es_rk_stage(ctx, 3, dt, JU, J, g2[0], g2[1], xt, xdt, *g3)
    assert es.es_check(ctx) == 0
    for (gu, gj), (ou, oj) in zip((g1, g2, g3), (o1, o2, o3)):
        assert rel_l1(to_np(gu), ou) < 1e-12
        assert rel_l1(to_np(gj), oj) < 1e-12


@pytest.mark.parametrize("case", ["sine1d", "riemann2d_ragged", "vortex_ideal", "rp1d_ragged"])
def test_cfl_parity(case):
    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    dt_o = stepper.cfl_dt(sch, JU_o, J_o, x, w["cfl"])
    dt_g = es.es_cfl_dt(ctx, JU, J, xt)
    assert abs(dt_g - dt_o) <= 1e-13 * dt_o


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["rp1d_ragged", "wavy_periodic"])
def test_cfl_with_mesh_velocity(case, precision):
    """eq. cfl with a mesh velocity in the spectral radius (|J xi_t + n . v| + |n| c, J xi_t = -xdot . n),
    against the oracle; the step's second time-step pass uses this form."""
    import torch

    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    xd = 10.0 * _xdot(w) if case == "wavy_periodic" else 2.0 * np.sin(2 * np.pi * w["x"])
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w, precision=precision)
    dt_o = stepper.cfl_dt(sch, JU_o, J_o, x, w["cfl"], xd)
    assert dt_o < 0.9 * stepper.cfl_dt(sch, JU_o, J_o, x, w["cfl"])
    dt_g = es.es_cfl_dt(ctx, JU, J, xt, torch.tensor(np.ascontiguousarray(xd), dtype=torch.float64, device="cuda"))
    assert abs(dt_g - dt_o) <= (1e-13 if precision == "fp64" else 1e-5) * dt_o


@pytest.mark.parametrize("case", ["riemann2d_ragged", "rp1d_ragged"])
def test_mesh_redistribution_parity(case):
    import torch

    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    dt = 0.004
    xdot_o, sw_o, gam_o = stepper.redistribute(sch, mc, JU_o, J_o, x, dt)
    xdot = torch.empty_like(xt)
    sw, gam = es.es_mesh_redistribute(ctx, JU, J, xt, dt, xdot)
    assert sw == sw_o
    assert abs(gam - gam_o) <= 1e-12 * max(gam_o, 1e-300)
    assert np.abs(to_np(xdot) - xdot_o).max() <= 1e-11 * np.abs(xdot_o).max()


def _one_step_compare(w, nsteps=1, t_end=None, tol=1e-12):
    from paper_2407_05568_gb300 import es
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    t_end = w["t_end"] if t_end is None else t_end
    t = 0.0
    for _ in range(nsteps):
        JU_o, J_o, x_o, t, info = stepper.step(sch, mc, JU_o, J_o, x_o, t, t_end, w["cfl"])
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, nsteps, t_end)
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    tg, dtg = es.es_get_time(ctx)
    assert abs(tg - t) <= 1e-12 * max(t, 1e-300)
    bound = tol * nsteps                      # the bar is 1e-12 relative L1 per step
    assert rel_l1(to_np(JU), JU_o) < bound
    assert rel_l1(to_np(J), J_o) < bound
    assert rel_l1(to_np(xt), x_o) < bound
    return ctx


def test_step_parity_sine1d():
    """Fixed-mesh 1D sine wave (200 nodes, CFL 0.4): 5 full steps."""
    _one_step_compare(wl.sine_1d(200), nsteps=5)


def test_step_parity_rp1d_moving():
    """Table 5.1 RP1 on a moving mesh (monitor with G, 10 sweeps): 3 steps."""
    _one_step_compare(_rp1d(300), nsteps=3)


def test_step_parity_riemann2d_ragged():
    _one_step_compare(_ragged_riemann(), nsteps=2)


@pytest.mark.parametrize("case", ["rp1d", "riemann2d_ragged"])
def test_step_parity_mm1(case):
    """The MM1 variant (monitor without G: alpha_2 = alpha_3 = 0) of Example 5.2's RP1 and of the 2D
    Riemann problem: 3 and 2 full steps."""
    w = wl.mm1(_rp1d(300) if case == "rp1d" else _ragged_riemann())
    _one_step_compare(w, nsteps=3 if case == "rp1d" else 2)


def test_step_parity_riemann2d_full_size():
    """The 200 x 200 moving-mesh vdW Riemann problem, in the launch configuration of the bench."""
    _one_step_compare(wl.riemann_2d(200, seed=5), nsteps=1)


def test_design_order_1d_sine_moving_mesh_gpu():
    """Example 5.1's MM on the GPU (smooth-test monitor, 20 filter passes, dt = CFL dxi^(5/3)): ~5th order
    in rho at the moved nodes, and the run at 80 nodes equals the oracle's."""
    from paper_2407_05568_gb300 import es
    errs = []
    for n in (20, 40, 80):
        w = wl.sine_1d(n, t_end=0.05, moving=True)
        dt = 0.4 * w["dxi"][0] ** (5.0 / 3.0)
        ctx, JU, J, xt = gpu_setup(w, dt_fixed=dt)
        es.es_set_time(ctx, 0.0)
        es.es_steps(ctx, JU, J, xt, int(np.ceil(w["t_end"] / dt)) + 2, w["t_end"])
        assert es.es_check(ctx) == 0, es.es_last_error(ctx)
        x = to_np(xt)
        ex = 0.5 + 0.2 * np.sin(2 * np.pi * (x[0] - w["t_end"]))
        errs.append(np.abs(to_np(JU)[0] / to_np(J) - ex).mean())
    order = np.log2(errs[-2] / errs[-1])
    assert order > 4.5, errs
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    JU_o, J_o, x_o, _ = stepper.run(sch, mc, JU_o, J_o, x_o, w["t_end"], 0.4, dt_fixed=dt)
    assert rel_l1(to_np(JU), JU_o) < 1e-10
    assert np.abs(x - x_o).max() < 1e-12


def test_es_step_is_one_of_es_steps():
    """es_step (one step, returning the time and the step taken) gives the bits of es_steps(1)."""
    from paper_2407_05568_gb300 import es
    w = _ragged_riemann()
    ctx1, JU1, J1, x1 = gpu_setup(w)
    ctx2, JU2, J2, x2 = gpu_setup(w)
    es.es_set_time(ctx1, 0.0)
    es.es_set_time(ctx2, 0.0)
    for _ in range(2):
        t, dt = es.es_step(ctx1, JU1, J1, x1, w["t_end"])
        es.es_steps(ctx2, JU2, J2, x2, 1, w["t_end"])
        assert (t, dt) == es.es_get_time(ctx2) and dt > 0.0
    assert es.es_check(ctx1) == 0 and es.es_check(ctx2) == 0
    assert np.array_equal(to_np(JU1), to_np(JU2)) and np.array_equal(to_np(x1), to_np(x2))


def test_steps_stop_at_t_end():
    """Steps after t_end are no-ops; the last step is shortened to land on t_end."""
    from paper_2407_05568_gb300 import es
    w = wl.sine_1d(64, t_end=0.01)
    ctx, JU, J, xt = gpu_setup(w)
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, 400, w["t_end"])
    t, _ = es.es_get_time(ctx)
    assert t == pytest.approx(0.01, rel=1e-14)
    before = to_np(JU).copy()
    es.es_steps(ctx, JU, J, xt, 3, w["t_end"])
    assert np.array_equal(to_np(JU), before)


def test_free_stream_gpu():
    """A constant state on a moving periodic mesh stays constant (Remark after eq. HOstable)."""
    import torch

    from paper_2407_05568_gb300 import es
    w = _wavy_periodic(32)
    X = w["x"][0]
    w["rho"] = np.full_like(X, 0.8)
    w["v"] = np.stack([np.full_like(X, 0.3), np.full_like(X, -0.2)])
    w["p"] = np.full_like(X, 1.1)
    ctx, JU, J, xt = gpu_setup(w)
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
    assert np.abs(to_np(JU) / to_np(J) - U0).max() < 1e-12 * np.abs(U0).max()


def test_run_host_matches_device_path():
    """es_run_host (host buffers, copies inside) gives the device path's result bit for bit."""
    from paper_2407_05568_gb300 import es
    w = _ragged_riemann()
    ctx, JU, J, xt = gpu_setup(w)
    hJU, hJ, hx = to_np(JU).copy(), to_np(J).copy(), to_np(xt).copy()
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, 2, w["t_end"])
    ctx2, _, _, _ = gpu_setup(w)
    es.es_set_time(ctx2, 0.0)
    es.es_run_host(ctx2, hJU, hJ, hx, 2, w["t_end"])
    assert np.array_equal(hJU, to_np(JU)) and np.array_equal(hJ, to_np(J)) and np.array_equal(hx, to_np(xt))


def test_inadmissible_state_is_reported():
    """A state outside eq. coefflimit (rho > 1/b) latches ES_ERR_INADMISSIBLE (host-made fault)."""
    import torch

    from paper_2407_05568_gb300 import es
    w = wl.sine_1d(64)
    w["rho"] = w["rho"].copy()
    w["rho"][17] = 3.2
    ctx, JU, J, xt = gpu_setup(w)
    dU = torch.empty_like(JU)
    dJ = torch.empty_like(J)
    es.es_rhs(ctx, JU, J, xt, None, dU, dJ)
    assert es.es_check(ctx) == es.ES_ERR_INADMISSIBLE
    assert "node 17" in es.es_last_error(ctx)
    assert es.es_check(ctx) == 0          # cleared after reading


def test_bad_parameters_rejected():
    from paper_2407_05568_gb300 import es
    w = wl.sine_1d(64)
    p = es.make_params(w)
    p.n1 = 4
    with pytest.raises(es.EsError):
        es.es_create(p)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["riemann2d_ragged", "wavy_rough"])
def test_tile_shapes_agree_bitwise(case, precision):
    """Every 2D tile shape gives the same operator (shapes only regroup nodes into CTAs): bit for bit
    in FP64, to FP32 rounding in the mixed form; and the autotuner picks one of them."""
    import torch

    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    xd = _xdot(w)
    xdt = torch.tensor(np.ascontiguousarray(xd), dtype=torch.float64, device="cuda")
    outs = []
    for tile in (1, 2, 3, 4, 5):
        from sides import gpu_setup as _gs
        p_ctx, JU, J, xt = _gs(w, precision=precision)
        ctx = es.es_create(es.make_params(w, precision=precision, tile=tile))
        dU = torch.empty_like(JU)
        dJ = torch.empty_like(J)
        es.es_rhs(ctx, JU, J, xt, xdt, dU, dJ)
        assert es.es_check(ctx) == 0
        outs.append((dU.clone(), dJ.clone()))
    for dU, dJ in outs[1:]:
        if precision == "fp64":
            assert torch.equal(dU, outs[0][0]) and torch.equal(dJ, outs[0][1])
        else:
            # FP32: each instantiation may fuse a different product of a sum into an FMA
            du = to_np(dU) - to_np(outs[0][0])
            assert np.abs(du).max() <= 1e-6 * np.abs(to_np(outs[0][0])).max(), np.abs(du).max()
    k, ms = es.es_autotune(p_ctx, JU, J, xt)
    assert k in (1, 2, 3, 4, 5) and all(m > 0 for m in ms)


def test_fp64_division_within_an_ulp_of_ieee():
    """The stage kernel's quotient and reciprocal (Newton-Raphson refined reciprocal, Markstein
    correction) against IEEE division, over magnitudes from 1e-12 to 1e12 and both signs."""
    import torch

    from paper_2407_05568_gb300 import es
    rng = np.random.default_rng(99)
    n = 1 << 20
    a = rng.standard_normal(n) * 10.0 ** rng.uniform(-12, 12, n)
    b = rng.standard_normal(n) * 10.0 ** rng.uniform(-12, 12, n)
    b[:8] = [1.0, -1.0, 3.0, 0.1, 1e-300 * 1e292, 7.0, 2.0 ** 52, 1.0 / 3.0]
    ta = torch.tensor(a, device="cuda")
    tb = torch.tensor(b, device="cuda")
    q = torch.empty_like(ta)
    r = torch.empty_like(ta)
    es.es_selftest_division(ta, tb, q, r)
    torch.cuda.synchronize()
    qn, rn = q.cpu().numpy(), r.cpu().numpy()
    assert np.all(np.abs(qn - a / b) <= np.spacing(np.abs(a / b)))
    assert np.all(np.abs(rn - 1.0 / b) <= np.spacing(np.abs(1.0 / b)))


def test_step_parity_jacobi_tolerance_graph_loop():
    """Jacobi to a tolerance inside the step graph (a while-loop node: one sweep per pass, the
    kernel ends the loop): two steps against the oracle, the same sweep counts."""
    from paper_2407_05568_gb300 import es
    w = _ragged_riemann()
    w["mesh"] = dict(w["mesh"], sweeps=40, eps=0.08 * w["dxi"][0])     # 24 and 23 sweeps: ends by tolerance
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    t = 0.0
    sweeps_o = 0
    for _ in range(2):
        JU_o, J_o, x_o, t, info = stepper.step(sch, mc, JU_o, J_o, x_o, t, w["t_end"], w["cfl"])
        sweeps_o += info["sweeps"]
    es.es_set_time(ctx, 0.0)
    es.es_mesh_stats(ctx, reset=True)
    es.es_steps(ctx, JU, J, xt, 2, w["t_end"])
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    sw, solves, _ = es.es_mesh_stats(ctx)
    assert solves == 2 and sw == sweeps_o and sw < 80
    assert rel_l1(to_np(JU), JU_o) < 2e-12
    assert rel_l1(to_np(xt), x_o) < 2e-12


def test_measured_alu_peaks():
    """The FMA-chain probe (the ALU roofline's denominators) reports rates of the right size for a GB300:
    FP32 near 152 SMs x 128 lanes x 2 x clock (~80 TFLOP/s at 2.07 GHz), FP64 near 1 TFLOP/s."""
    from paper_2407_05568_gb300 import es
    f64, f32 = es.es_selftest_peaks()
    assert 40.0 < f32 < 100.0, f32
    assert 0.4 < f64 < 2.5, f64
    assert f32 > 30.0 * f64


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_time_stage(precision):
    """es_time_stage times back-to-back launches of the stage kernel es_rk_stage runs: a positive time per
    launch, no device error, and ES_ERR_ARG for bad arguments."""
    import torch

    from paper_2407_05568_gb300 import es
    w = wl.riemann_2d(64, seed=5)
    ctx, JU, J, xt = gpu_setup(w, precision=precision)
    ms = es.es_time_stage(ctx, JU, J, xt, stage=2, dt=1e-4, reps=5)
    assert 0.0 < ms < 50.0, ms
    assert es.es_check(ctx) == 0
    with pytest.raises(es.EsError):
        es.es_time_stage(ctx, JU, J, xt, stage=4)
    with pytest.raises(es.EsError):
        es.es_time_stage(ctx, JU, J, xt, reps=0)
