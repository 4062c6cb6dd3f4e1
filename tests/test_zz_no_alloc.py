"""The allocation-free SSP-RK3 step against the context-based stage calls.

es_rk3_step_static serves callers that cannot allocate device memory: it keeps
its two stage states in a fixed array compiled into the library.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2407_05568_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_05568_gb300 import build
    build.build()


def _problem(case):
    if case == "riemann2d":
        w = wl.riemann_2d(8, seed=3)
        x1, d1 = wl.uniform_nodes(70, 0.0, 1.0, False)
        x2, d2 = wl.uniform_nodes(45, 0.0, 1.0, False)
        X, Y = np.meshgrid(x1, x2)
        st = np.array(wl.quadrant_states(3))
        q = np.where(X > 0.5, np.where(Y > 0.5, 0, 3), np.where(Y > 0.5, 1, 2))
        w.update(n=(45, 70), dxi=(d1, d2), x=np.stack([X, Y]), rho=st[q, 0],
                 v=np.stack([st[q, 1], st[q, 2]]), p=st[q, 3])
        w["xdot"] = wl.mesh_velocity_2d(X, Y, amp=0.01, fixed_edges=True)
        return w
    w = wl.riemann_1d("RP1", n=300)
    w["xdot"] = np.zeros_like(w["x"])
    return w


@pytest.mark.parametrize("case", ["riemann2d", "rp1d"])
def test_static_step_matches_context_stages(case):
    import torch

    from paper_2407_05568_gb300 import es
    w = _problem(case)
    dev = torch.device("cuda:0")
    params = es.make_params(w)
    ctx = es.es_create(params)
    x = torch.tensor(w["x"], dtype=torch.float64, device=dev)
    xdot = torch.tensor(w["xdot"], dtype=torch.float64, device=dev)
    J0 = torch.empty(w["x"].shape[1:], dtype=torch.float64, device=dev)
    es.es_init_mesh(ctx, x, J0)
    JU0 = torch.empty((w["dim"] + 2,) + w["x"].shape[1:], dtype=torch.float64, device=dev)
    es.es_prim_to_cons(ctx, torch.tensor(w["rho"], device=dev), torch.tensor(w["v"], device=dev),
                       torch.tensor(w["p"], device=dev), J0, JU0)
    dt = 0.2 * min(w["dxi"])
    # reference: two steps through the existing context-based entry point
    JU_ref, J_ref = JU0.clone(), J0.clone()
    a = (torch.empty_like(JU0), torch.empty_like(J0))
    b = (torch.empty_like(JU0), torch.empty_like(J0))
    refs = []
    for _ in range(2):
        es.es_rk_stage(ctx, 1, dt, JU_ref, J_ref, JU_ref, J_ref, x, xdot, *a)
        es.es_rk_stage(ctx, 2, dt, JU_ref, J_ref, a[0], a[1], x, xdot, *b)
        es.es_rk_stage(ctx, 3, dt, JU_ref, J_ref, b[0], b[1], x, xdot, JU_ref, J_ref)
        refs.append((JU_ref.clone(), J_ref.clone()))
    assert es.es_check(ctx) == 0
    # the allocation-free entry point, two calls in a row on the same arrays
    JU, J = JU0.clone(), J0.clone()
    torch.cuda.synchronize()
    for k in range(2):
        rc = es.es_rk3_step_static(params, dt, JU, J, x, xdot)
        assert rc == 0
        for got, ref in ((JU, refs[k][0]), (J, refs[k][1])):
            g = got.cpu().numpy()
            r = ref.cpu().numpy()
            assert np.abs(g - r).sum() / np.abs(r).sum() < 1e-12


def test_static_step_allocates_nothing_after_its_first_call():
    """After the first call on the device (its set-up), further calls leave the device's free memory unchanged,
    on the default stream and on another stream, and give the same result on both."""
    import torch

    from paper_2407_05568_gb300 import es
    w = _problem("riemann2d")
    dev = torch.device("cuda:0")
    params = es.make_params(w)
    ctx = es.es_create(params)
    x = torch.tensor(w["x"], dtype=torch.float64, device=dev)
    xdot = torch.tensor(w["xdot"], dtype=torch.float64, device=dev)
    J = torch.empty(w["x"].shape[1:], dtype=torch.float64, device=dev)
    es.es_init_mesh(ctx, x, J)
    JU = torch.empty((w["dim"] + 2,) + w["x"].shape[1:], dtype=torch.float64, device=dev)
    es.es_prim_to_cons(ctx, torch.tensor(w["rho"], device=dev), torch.tensor(w["v"], device=dev),
                       torch.tensor(w["p"], device=dev), J, JU)
    JU2, J2 = JU.clone(), J.clone()
    side = torch.cuda.Stream()
    dt = 0.2 * min(w["dxi"])
    torch.cuda.synchronize()
    assert es.es_rk3_step_static(params, dt, JU, J, x, xdot) == 0          # set-up call
    free0, _ = torch.cuda.mem_get_info()
    assert es.es_rk3_step_static(params, dt, JU, J, x, xdot) == 0
    free1, _ = torch.cuda.mem_get_info()
    assert es.es_rk3_step_static(params, dt, JU2, J2, x, xdot, stream=side) == 0
    assert es.es_rk3_step_static(params, dt, JU2, J2, x, xdot, stream=side) == 0
    free2, _ = torch.cuda.mem_get_info()
    assert free0 == free1 == free2
    assert torch.equal(JU, JU2) and torch.equal(J, J2)


def test_static_step_rejects_large_meshes():
    from paper_2407_05568_gb300 import es
    w = wl.sine_2d(300)                          # 90000 nodes > 65536
    p = es.make_params(w)
    import torch
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert es.es_rk3_step_static(p, 1e-3, t, t, t) == es.ES_ERR_ARG
