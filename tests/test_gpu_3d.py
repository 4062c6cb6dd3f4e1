"""Parity of the 3D CUDA path with the FP64 oracle (Sec. 3 - Sec. 4 in three dimensions).

Meshes have three different sizes (so a swapped axis shows), more nodes along xi_1 than one
pencil (16) holds and ragged pencils in every direction; periodic wavy meshes with a
mesh velocity, outflow boundaries, walls, and the spherical shock tube geometry of Example 5.7
with symmetry planes through the centre and the moving mesh.  Bar: 1e-12 relative per step, as in
1D/2D.
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


def _box(n1, n2, n3, periodic, amp=0.0, seed=None):
    """A 3D workload on [0,1]^3 with sizes (n1, n2, n3), an optional wavy mesh and a smooth or
    seeded rough state."""
    tp = 2 * np.pi
    ax = [wl.uniform_nodes(n, 0.0, 1.0, periodic) for n in (n1, n2, n3)]
    Z, Y, X = np.meshgrid(ax[2][0], ax[1][0], ax[0][0], indexing="ij")
    x = np.stack([X + amp * np.sin(tp * X) * np.sin(tp * Y) * np.cos(tp * Z),
                  Y + amp * np.sin(tp * Y) * np.cos(tp * X) * np.sin(tp * Z),
                  Z + amp * np.sin(tp * Z) * np.sin(tp * X + 0.3) * np.sin(tp * Y)])
    if seed is None:
        # phases off the node grid (at an exact symmetric extremum the MR-WENO5 weights turn on
        # the last bits of W, in the oracle as much as here)
        rho = 0.6 + 0.15 * np.sin(tp * X + 0.37) * np.cos(tp * Y + 0.21) + 0.05 * np.sin(tp * Z + 0.13)
        v = np.stack([0.3 + 0.1 * np.cos(tp * Y + 0.29), -0.2 + 0.1 * np.sin(tp * Z + 0.41),
                      0.1 + 0.1 * np.sin(tp * X + 0.17)])
        p = 1.0 + 0.1 * np.sin(tp * (Y + Z) + 0.23)
    else:
        rng = np.random.default_rng(seed)
        rho = 0.7 + 0.4 * rng.uniform(size=X.shape)
        v = 0.3 * rng.standard_normal((3,) + X.shape)
        p = 1.0 + 0.4 * rng.uniform(size=X.shape)
    bc = "periodic" if periodic else "outflow"
    return dict(gas=wl.UNITS_A, dim=3, n=(n3, n2, n1), dxi=(ax[0][1], ax[1][1], ax[2][1]), bc=(bc,) * 3,
                period=(1.0, 1.0, 1.0), x=x, rho=rho, v=v, p=p, t_end=1.0, cfl=0.4, moving=False)


def _shock(n1, n2, n3):
    """Example 5.7's geometry with two supercritical states (T = 1.15 inside, 1.04 outside).  The
    Table 5.1 states put face states next to the spinodal on meshes this coarse, where the
    entropy-wave scaling (R T - 2 a rho (1 - b rho)^2)^(-1/2) turns rounding into 1e-10 changes."""
    w = wl.spherical_shock_3d(8)
    ax = [wl.uniform_nodes(n, 0.0, 1.0, False) for n in (n1, n2, n3)]
    Z, Y, X = np.meshgrid(ax[2][0], ax[1][0], ax[0][0], indexing="ij")
    inside = X**2 + Y**2 + Z**2 < 0.25
    w.update(n=(n3, n2, n1), dxi=(ax[0][1], ax[1][1], ax[2][1]), x=np.stack([X, Y, Z]),
             rho=np.where(inside, 1.2, 0.6), v=np.zeros((3,) + X.shape), p=np.where(inside, 1.8, 1.0))
    return w


CASES = {
    "wavy_periodic_smooth": lambda: _box(20, 18, 17, True, amp=0.01),
    "wavy_periodic_rough": lambda: _box(19, 22, 12, True, amp=0.01, seed=4),
    "outflow_rough": lambda: _box(18, 12, 21, False, amp=0.0, seed=9),
    "shock_ragged": lambda: _shock(19, 17, 21),          # symmetry planes at x_k = 0, outflow at 1
    "walls_rough": lambda: dict(_box(17, 20, 19, False, amp=0.0, seed=13), bc=("reflect",) * 3),
}


def _xdot(w):
    tp = 2 * np.pi
    X, Y, Z = w["x"]
    return 0.05 * np.stack([np.sin(tp * (X + Y)), np.cos(tp * (Y - Z)), np.sin(tp * (Z + X))])


@pytest.mark.parametrize("case", list(CASES))
def test_init_parity_3d(case):
    w = CASES[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    assert rel_l1(to_np(J), J_o) < 1e-14
    assert rel_l1(to_np(JU), JU_o) < 1e-14


@pytest.mark.parametrize("dissipation", [True, False])
@pytest.mark.parametrize("case", list(CASES))
def test_rhs_parity_3d(case, dissipation):
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
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    scale = np.abs(JU_o).sum() / min(w["dxi"])
    err = np.abs(to_np(dU) - dU_o).sum() / scale
    assert err < 1e-12, err
    errJ = np.abs(to_np(dJ) - dJ_o).sum() / (np.abs(J_o).sum() / min(w["dxi"]))
    assert errJ < 1e-12, errJ
    assert np.abs(dU_o).sum() > 1e-6 * scale * min(w["dxi"])


@pytest.mark.parametrize("case", ["wavy_periodic_rough", "shock_ragged", "walls_rough"])
def test_rk_stage_parity_3d(case):
    import torch

    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    xd = _xdot(w)
    xdt = torch.tensor(np.ascontiguousarray(xd), dtype=torch.float64, device="cuda")
    dt = 0.5 * stepper.cfl_dt(sch, JU_o, J_o, x, w["cfl"])
    o1 = stepper.rk_stage(sch, 0, dt, JU_o, J_o, JU_o, J_o, x, xd)
    o2 = stepper.rk_stage(sch, 1, dt, JU_o, J_o, o1[0], o1[1], x, xd)
    o3 = stepper.rk_stage(sch, 2, dt, JU_o, J_o, o2[0], o2[1], x, xd)
    g = [(torch.empty_like(JU), torch.empty_like(J)) for _ in range(3)]
    es.es_rk_stage(ctx, 1, dt, JU, J, JU, J, xt, xdt, *g[0])
    es.es_rk_stage(ctx, 2, dt, JU, J, g[0][0], g[0][1], xt, xdt, *g[1])
    es.es_rk_stage(ctx, 3, dt, JU, J, g[1][0], g[1][1], xt, xdt, *g[2])
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    for (gu, gj), (ou, oj) in zip(g, (o1, o2, o3)):
        assert rel_l1(to_np(gu), ou) < 1e-12
        assert rel_l1(to_np(gj), oj) < 1e-12


@pytest.mark.parametrize("case", ["wavy_periodic_smooth", "outflow_rough", "shock_ragged"])
def test_cfl_parity_3d(case):
    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    dt_o = stepper.cfl_dt(sch, JU_o, J_o, x, w["cfl"])
    dt_g = es.es_cfl_dt(ctx, JU, J, xt)
    assert abs(dt_g - dt_o) <= 1e-13 * dt_o


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cfl_with_mesh_velocity_3d(precision):
    """eq. cfl with a mesh velocity in the spectral radius (|J xi_t + n . v| + |n| c), against the oracle."""
    import torch

    from paper_2407_05568_gb300 import es
    w = CASES["wavy_periodic_smooth"]()
    X, Y, Z = w["x"]
    tp = 2 * np.pi
    xd = 0.8 * np.stack([np.sin(tp * (X + Y)), np.cos(tp * (Y - Z)), np.sin(tp * (Z + X))])
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w, precision=precision)
    dt_o = stepper.cfl_dt(sch, JU_o, J_o, x, w["cfl"], xd)
    assert dt_o < 0.9 * stepper.cfl_dt(sch, JU_o, J_o, x, w["cfl"])          # the mesh velocity matters here
    dt_g = es.es_cfl_dt(ctx, JU, J, xt, torch.tensor(xd, dtype=torch.float64, device="cuda"))
    assert abs(dt_g - dt_o) <= (1e-13 if precision == "fp64" else 1e-5) * dt_o


def _moving(w, monitor="vdw"):
    w = dict(w, moving=True)
    if monitor == "vdw":
        w["mesh"] = dict(monitor="vdw", alphas=(1200.0, 1200.0, 0.0), kappa=2, filter_passes=3, sweeps=6, eps=0.0)
    else:
        w["mesh"] = dict(monitor="smooth", alphas=(20.0, 15.0), kappa=2, filter_passes=2, sweeps=6, eps=0.0)
    return w


@pytest.mark.parametrize("case,monitor", [("shock_ragged", "vdw"), ("wavy_periodic_smooth", "smooth"),
                                          ("outflow_rough", "vdw"), ("walls_rough", "vdw")])
def test_mesh_redistribution_parity_3d(case, monitor):
    import torch

    from paper_2407_05568_gb300 import es
    w = _moving(CASES[case](), monitor)
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    dt = 0.002
    xdot_o, sw_o, gam_o = stepper.redistribute(sch, mc, JU_o, J_o, x, dt)
    xdot = torch.empty_like(xt)
    sw, gam = es.es_mesh_redistribute(ctx, JU, J, xt, dt, xdot)
    assert sw == sw_o
    assert abs(gam - gam_o) <= 1e-12 * max(gam_o, 1e-300)
    assert np.abs(xdot_o).max() > 0.0
    assert np.abs(to_np(xdot) - xdot_o).max() <= 1e-11 * np.abs(xdot_o).max()


@pytest.mark.parametrize("case,monitor,nsteps", [("shock_ragged", "vdw", 2), ("wavy_periodic_smooth", "smooth", 2),
                                                 ("wavy_periodic_rough", None, 1), ("walls_rough", "vdw", 1),
                                                 ("outflow_rough", "vdw", 2)])
def test_step_parity_3d(case, monitor, nsteps):
    """Full steps through es_steps (CFL, mesh redistribution, three stages; a CUDA graph)."""
    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    if monitor:
        w = _moving(w, monitor)
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    t = 0.0
    for _ in range(nsteps):
        JU_o, J_o, x_o, t, _ = stepper.step(sch, mc, JU_o, J_o, x_o, t, w["t_end"], w["cfl"])
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, nsteps, w["t_end"])
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    tg, _ = es.es_get_time(ctx)
    assert abs(tg - t) <= 1e-12 * t
    bound = 1e-12 * nsteps
    assert rel_l1(to_np(JU), JU_o) < bound
    assert rel_l1(to_np(J), J_o) < bound
    assert rel_l1(to_np(xt), x_o) < bound


def test_rhs_parity_3d_48():
    """A larger periodic wavy mesh (48 x 40 x 36: three pencils along xi_1) against the oracle."""
    import torch

    from paper_2407_05568_gb300 import es
    w = _box(48, 40, 36, True, amp=0.01, seed=21)
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    xd = _xdot(w)
    dU_o, dJ_o = op.rhs(sch, JU_o, J_o, x, xd)
    xdt = torch.tensor(np.ascontiguousarray(xd), dtype=torch.float64, device="cuda")
    dU = torch.empty_like(JU)
    dJ = torch.empty_like(J)
    es.es_rhs(ctx, JU, J, xt, xdt, dU, dJ)
    assert es.es_check(ctx) == 0
    scale = np.abs(JU_o).sum() / min(w["dxi"])
    assert np.abs(to_np(dU) - dU_o).sum() / scale < 1e-12


def test_free_stream_3d_gpu_full_size():
    """At 100^3 (outflow, a wavy interior mesh moving) a constant state stays constant:
    d(JU)/dt = U dJ/dt to round-off (the oracle cannot run this size in seconds)."""
    import torch

    from paper_2407_05568_gb300 import es
    w = _box(100, 100, 100, False, amp=0.0)
    X, Y, Z = w["x"]
    tp = 2 * np.pi
    bump = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    w["x"] = np.stack([X + 0.003 * bump * np.sin(tp * Y), Y + 0.003 * bump * np.sin(tp * Z),
                       Z + 0.003 * bump * np.sin(tp * X)])
    w["rho"] = np.full_like(X, 0.8)
    w["v"] = np.stack([0.3 + 0 * X, -0.2 + 0 * X, 0.1 + 0 * X])
    w["p"] = np.full_like(X, 1.1)
    ctx, JU, J, xt = gpu_setup(w)
    xd = torch.tensor(0.05 * bump * np.stack([np.sin(tp * Y), np.cos(tp * Z), np.sin(tp * X)]),
                      dtype=torch.float64, device="cuda")
    dU = torch.empty_like(JU)
    dJ = torch.empty_like(J)
    es.es_rhs(ctx, JU, J, xt, xd, dU, dJ)
    assert es.es_check(ctx) == 0
    U0 = (JU / J).cpu().numpy()
    res = to_np(dU) - U0 * to_np(dJ)
    assert np.abs(res).max() < 1e-12 * np.abs(U0).max() / min(w["dxi"])
    assert np.abs(to_np(dJ)).max() > 1e-3


def test_3d_rejections():
    """Walls in the mixed form and the 2D-only calls refuse a 3D context with ES_ERR_ARG."""
    import ctypes

    from paper_2407_05568_gb300 import es
    w = CASES["walls_rough"]()
    p = es.make_params(w, precision="mixed")
    h = ctypes.c_void_p()
    assert es.lib().es_create(ctypes.byref(h), ctypes.byref(p), None) == es.ES_ERR_ARG
    w = CASES["wavy_periodic_smooth"]()
    ctx, JU, J, xt = gpu_setup(w)
    with pytest.raises(es.EsError):
        es.es_mesh_solve(ctx, JU, J, xt, None, xt.clone())


def test_pencil_shapes_agree_bitwise_and_autotune():
    """The pencil shapes of the 3D direction kernels group faces differently but evaluate each face
    the same way: identical bits; the autotuner picks one of them."""
    import torch

    from paper_2407_05568_gb300 import es
    w = CASES["wavy_periodic_rough"]()
    outs = []
    for tile in (1, 2, 3, 4):
        p = es.make_params(w, tile=tile)
        ctx = es.es_create(p)
        xt = torch.tensor(w["x"], dtype=torch.float64, device="cuda")
        J = torch.empty(w["x"].shape[1:], dtype=torch.float64, device="cuda")
        es.es_init_mesh(ctx, xt, J)
        JU = torch.empty((5,) + w["x"].shape[1:], dtype=torch.float64, device="cuda")
        es.es_prim_to_cons(ctx, torch.tensor(w["rho"], device="cuda"), torch.tensor(w["v"], device="cuda"),
                           torch.tensor(w["p"], device="cuda"), J, JU)
        xd = torch.tensor(np.ascontiguousarray(_xdot(w)), dtype=torch.float64, device="cuda")
        dU, dJ = torch.empty_like(JU), torch.empty_like(J)
        es.es_rhs(ctx, JU, J, xt, xd, dU, dJ)
        assert es.es_check(ctx) == 0
        outs.append((dU.cpu().numpy(), dJ.cpu().numpy()))
    for o in outs[1:]:
        assert np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1])
    ctx, JU, J, xt = gpu_setup(w)
    k, ms = es.es_autotune(ctx, JU, J, xt)
    assert k in (1, 2, 3, 4) and all(m > 0 for m in ms[:4])


def _mixed_rhs(w, tile):
    """Right-hand sides of the mixed form's 3D operator with the given tile (pencil shape) parameter."""
    import torch

    from paper_2407_05568_gb300 import es
    ctx = es.es_create(es.make_params(w, precision="mixed", tile=tile))
    shape = w["x"].shape[1:]
    xt = torch.tensor(w["x"], dtype=torch.float64, device="cuda")
    J = es.state_empty(ctx, shape, "cuda")
    es.es_init_mesh(ctx, xt, J)
    JU = es.state_empty(ctx, (5,) + shape, "cuda")
    es.es_prim_to_cons(ctx, torch.tensor(w["rho"], device="cuda"), torch.tensor(w["v"], device="cuda"),
                       torch.tensor(w["p"], device="cuda"), J, JU)
    xd = torch.tensor(np.ascontiguousarray(_xdot(w)), dtype=torch.float64, device="cuda")
    dU, dJ = torch.empty_like(JU), torch.empty_like(J)
    es.es_rhs(ctx, JU, J, xt, xd, dU, dJ)
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    return dU.cpu().numpy(), dJ.cpu().numpy()


@pytest.mark.parametrize("n,periodic,seed", [((20, 18, 17), True, 4), ((24, 12, 21), False, 9),
                                             ((64, 40, 36), True, None)])
def test_mixed_3d_tma_staging_matches_plain_loads_bitwise(n, periodic, seed):
    """The xi_2 and xi_3 direction kernels of the mixed form stage a pencil's node fields with one TMA copy
    (persistent CTAs, the next pencil's copy in flight during the current one; n1 a multiple of 4) or load them
    node by node (tiles 5..8: shapes 1..4 without the staging).  The same floats reach shared memory, so the
    right-hand sides agree bit for bit for every pencil shape: on ragged meshes whose pencils have ghost rows
    (periodic wrap, outflow copy) and lines past the mesh, and on 64 x 40 x 36, where a CTA takes several
    pencils."""
    w = _box(*n, periodic, amp=0.01 if periodic else 0.0, seed=seed)
    for tile in (1, 2, 3, 4):
        a = _mixed_rhs(w, tile)
        b = _mixed_rhs(w, tile + 4)
        assert np.isfinite(a[0]).all()
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), tile


# ------------------------------------------------------------------ mixed form
def _mixed_case(case):
    w = CASES[case]()
    if case == "shock_ragged":                   # the mixed form has periodic and outflow ends only
        w = dict(w, bc=("outflow",) * 3)
    return w


@pytest.mark.parametrize("case", ["wavy_periodic_smooth", "wavy_periodic_rough", "outflow_rough", "shock_ragged"])
def test_mixed_3d_rhs_against_oracle(case):
    """The mixed form's 3D operator (FP32 direction kernels, double-float node values and jumps)
    within 1e-5 of the flux scale of the FP64 oracle (5.2e-6 measured on the shock state with the MR-WENO epsilon of
    1e-6; 2.5e-6 with 1e-12)."""
    import torch

    from paper_2407_05568_gb300 import es
    w = _mixed_case(case)
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w, precision="mixed")
    xd = _xdot(w)
    dU_o, dJ_o = op.rhs(sch, JU_o, J_o, x, xd)
    dU, dJ = torch.empty_like(JU), torch.empty_like(J)
    es.es_rhs(ctx, JU, J, xt, torch.tensor(np.ascontiguousarray(xd), device="cuda"), dU, dJ)
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    scale = np.abs(JU_o).sum() / min(w["dxi"])
    err = np.abs(to_np(dU) - dU_o).sum() / scale
    assert err < 1e-5, err
    assert np.abs(to_np(dJ) - dJ_o).sum() / (np.abs(J_o).sum() / min(w["dxi"])) < 1e-5


@pytest.mark.parametrize("case,monitor", [("wavy_periodic_smooth", "smooth"), ("shock_ragged", "vdw")])
def test_mixed_3d_steps_against_oracle(case, monitor):
    """Two full moving-mesh steps of the mixed form against the FP64 oracle: within 2e-6 (relative L1)."""
    from paper_2407_05568_gb300 import es
    w = _moving(_mixed_case(case), monitor)
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w, precision="mixed")
    t = 0.0
    for _ in range(2):
        JU_o, J_o, x_o, t, _ = stepper.step(sch, mc, JU_o, J_o, x_o, t, w["t_end"], w["cfl"])
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, 2, w["t_end"])
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    assert rel_l1(to_np(JU), JU_o) < 2e-6, rel_l1(to_np(JU), JU_o)
    assert rel_l1(to_np(xt), x_o) < 1e-6


@pytest.mark.parametrize("case,monitor,eps", [("shock_ragged", "vdw", 0.0), ("wavy_periodic_smooth", "smooth", 0.0),
                                              ("outflow_rough", "vdw", 0.0), ("outflow_rough", "vdw", 1e30)])
def test_mixed_3d_mesh_redistribution_against_oracle(case, monitor, eps):
    """The mixed form's mesh redistribution (FP32 monitor, filter and sweeps on the displacement from
    x^n): the same sweeps, Delta_gamma and mesh velocity as the FP64 oracle to FP32 rounding.  A
    tolerance of 1e30 stops the iteration after its first sweep on both sides."""
    import torch

    from paper_2407_05568_gb300 import es
    w = _moving(_mixed_case(case), monitor)
    w["mesh"]["eps"] = eps
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w, precision="mixed")
    dt = 0.002
    xdot_o, sw_o, gam_o = stepper.redistribute(sch, mc, JU_o, J_o, x, dt)
    xdot = torch.empty_like(xt)
    sw, gam = es.es_mesh_redistribute(ctx, JU, J, xt, dt, xdot)
    assert sw == sw_o == (1 if eps > 0 else w["mesh"]["sweeps"])
    assert abs(gam - gam_o) <= 1e-5 * gam_o
    assert np.abs(xdot_o).max() > 0.0
    assert np.abs(to_np(xdot) - xdot_o).max() <= 2e-5 * np.abs(xdot_o).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_run_host_3d_matches_device_path(prec):
    """es_run_host on a 3D context (host buffers, copies inside) gives the device path's bits, both forms."""
    from paper_2407_05568_gb300 import es
    w = _moving(_mixed_case("wavy_periodic_smooth"), "smooth")
    ctx, JU, J, xt = gpu_setup(w, precision=prec)
    hJU, hJ, hx = JU.cpu().numpy().copy(), J.cpu().numpy().copy(), xt.cpu().numpy().copy()
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, 2, w["t_end"])
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    ctx2, _, _, _ = gpu_setup(w, precision=prec)
    es.es_set_time(ctx2, 0.0)
    es.es_run_host(ctx2, hJU, hJ, hx, 2, w["t_end"])
    assert es.es_check(ctx2) == 0, es.es_last_error(ctx2)
    assert np.array_equal(hJU, JU.cpu().numpy()) and np.array_equal(hJ, J.cpu().numpy())
    assert np.array_equal(hx, xt.cpu().numpy())


@pytest.mark.parametrize("periodic,prec", [(True, "fp64"), (False, "fp64"), (True, "mixed"), (False, "mixed")])
def test_smallest_3d_mesh_against_oracle(periodic, prec):
    """The smallest mesh a 3D context accepts (8 nodes in every direction: the 3-node halos and the
    pencils' ghosts wrap or reflect across most of the mesh): one moving-mesh step against the oracle."""
    from paper_2407_05568_gb300 import es
    w = _moving(_box(8, 8, 8, periodic, amp=0.01 if periodic else 0.0, seed=21), "vdw")
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    JU_o, J_o, x_o, t, _ = stepper.step(sch, mc, JU_o, J_o, x_o, 0.0, w["t_end"], w["cfl"])
    ctx, JU, J, xt = gpu_setup(w, precision=prec)
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, 1, w["t_end"])
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    bound = 1e-12 if prec == "fp64" else 2e-6
    assert rel_l1(to_np(JU), JU_o) < bound, rel_l1(to_np(JU), JU_o)
    assert np.abs(to_np(xt) - x_o).max() < (1e-12 if prec == "fp64" else 1e-6)


def test_mixed_3d_sine_to_final_time_against_fp64():
    """The 3D sine wave (Example 5.6 setup, fixed mesh) at 40^3 to t = 0.05: the mixed form stays within
    1e-5 (relative L1) of the FP64 path, whose error against the exact solution it matches."""
    from paper_2407_05568_gb300 import es
    w = wl.sine_3d(40, t_end=0.05)
    res = {}
    for prec in ("fp64", "mixed"):
        ctx, JU, J, xt = gpu_setup(w, precision=prec)
        es.es_set_time(ctx, 0.0)
        es.es_steps(ctx, JU, J, xt, 400, w["t_end"])
        assert es.es_check(ctx) == 0, es.es_last_error(ctx)
        t, _ = es.es_get_time(ctx)
        assert abs(t - w["t_end"]) < 1e-12
        res[prec] = to_np(JU)[0] / to_np(J)
    X, Y, Z = w["x"]
    exact = 0.5 + 0.2 * np.sin(2 * np.pi * (X + Y + Z - 0.9 * w["t_end"]))
    assert rel_l1(res["mixed"], res["fp64"]) < 1e-5
    e64, e32 = np.abs(res["fp64"] - exact).mean(), np.abs(res["mixed"] - exact).mean()
    assert e32 < 1.5 * e64 + 1e-6, (e64, e32)


def test_design_order_3d_sine_moving_mesh():
    """Example 5.6: the 3D sine wave on the moving mesh (Example 5.1's monitor and 20 filter passes, MR-WENO linear
    weights 1/3 each) to t = 0.1 with dt = 0.3 dxi^(5/3) (Example 5.1's rule, so the spatial error dominates), in FP64.
    The error in rho at the moved nodes falls at fifth order or better from 48^3 to 64^3 to 96^3 (coarser meshes are
    not yet in the asymptotic range of this diagonal wave: with these linear weights the nonlinear weights approach
    them only once the smoothness indicators exceed epsilon), and the 16^3 run equals the oracle's."""
    from paper_2407_05568_gb300 import es
    errs = []
    sizes = (16, 48, 64, 96)
    for n in sizes:
        w = wl.sine_3d(n, t_end=0.1, moving=True)
        dt = 0.3 * w["dxi"][0] ** (5.0 / 3.0)
        ctx, JU, J, xt = gpu_setup(w, dt_fixed=dt)
        es.es_set_time(ctx, 0.0)
        es.es_steps(ctx, JU, J, xt, int(np.ceil(w["t_end"] / dt)) + 2, w["t_end"])
        assert es.es_check(ctx) == 0, es.es_last_error(ctx)
        assert es.es_get_time(ctx)[0] == pytest.approx(w["t_end"], rel=1e-12)
        x = to_np(xt)
        assert np.abs(x - w["x"]).max() > 1e-3 * w["dxi"][0]                 # the mesh moved
        exact = 0.5 + 0.2 * np.sin(2 * np.pi * (x[0] + x[1] + x[2] - 0.9 * w["t_end"]))
        errs.append(np.abs(to_np(JU)[0] / to_np(J) - exact).mean())
        if n == 16:
            sch, mc, JU_o, J_o, x_o = oracle_setup(w)
            JU_o, J_o, x_o, _ = stepper.run(sch, mc, JU_o, J_o, x_o, w["t_end"], w["cfl"], dt_fixed=dt)
            assert rel_l1(to_np(JU), JU_o) < 1e-11
            assert np.abs(x - x_o).max() < 1e-12
    orders = [np.log(errs[i] / errs[i + 1]) / np.log(sizes[i + 1] / sizes[i]) for i in range(1, len(sizes) - 1)]
    assert orders[-1] > 4.5 and orders[-2] > 4.5, (errs, orders)
