"""Walls and symmetry planes in the 1D/2D FP64 kernels against the oracle (the oracle's boundary
rule is pinned by the half and quarter problems reproducing the full mirror-symmetric ones).

Cases: a 1D shock tube with a wall at both ends, a 2D quarter of a circular Riemann problem with
symmetry planes at x = 0 and y = 0 (outflow at 1), and a 2D box with walls and a rough state.
Bar: 1e-12 relative per step.
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


MESH = dict(monitor="vdw", alphas=(1200.0, 1200.0, 1200.0), kappa=2, filter_passes=3, sweeps=5, eps=0.0)


def _tube_walls():
    x, d = wl.uniform_nodes(70, 0.0, 1.0, False)
    left = x < 0.37
    return dict(gas=wl.UNITS_A, dim=1, n=(70,), dxi=(d,), bc=("reflect",), period=(1.0,), x=x[None].copy(),
                rho=np.where(left, 1.2, 0.6), v=np.where(left, 0.2, -0.1)[None], p=np.where(left, 1.8, 1.0),
                t_end=1.0, cfl=0.4, moving=True, mesh=MESH)


def _quarter():
    a1, d1 = wl.uniform_nodes(33, 0.0, 1.0, False)
    a2, d2 = wl.uniform_nodes(26, 0.0, 1.0, False)
    Y, X = np.meshgrid(a2, a1, indexing="ij")
    r2 = X**2 + Y**2
    inside = r2 < 0.17
    v = np.stack([0.2 * X * np.exp(-r2), 0.2 * Y * np.exp(-r2)])
    return dict(gas=wl.UNITS_A, dim=2, n=(26, 33), dxi=(d1, d2), bc=("symmetry_lo", "symmetry_lo"),
                period=(1.0, 1.0), x=np.stack([X, Y]), rho=np.where(inside, 1.2, 0.6) + 0.05 * np.exp(-10 * r2),
                v=v, p=np.where(inside, 1.8, 1.0), t_end=1.0, cfl=0.4, moving=True, mesh=MESH)


def _box_walls():
    a1, d1 = wl.uniform_nodes(29, 0.0, 1.0, False)
    a2, d2 = wl.uniform_nodes(22, 0.0, 1.0, False)
    Y, X = np.meshgrid(a2, a1, indexing="ij")
    rng = np.random.default_rng(17)
    return dict(gas=wl.UNITS_A, dim=2, n=(22, 29), dxi=(d1, d2), bc=("reflect", "reflect"), period=(1.0, 1.0),
                x=np.stack([X, Y]), rho=0.7 + 0.4 * rng.uniform(size=X.shape),
                v=0.3 * rng.standard_normal((2,) + X.shape), p=1.0 + 0.4 * rng.uniform(size=X.shape),
                t_end=1.0, cfl=0.4, moving=True, mesh=MESH)


CASES = {"tube_walls": _tube_walls, "quarter_symmetry": _quarter, "box_walls": _box_walls}


def _xdot(w):
    if w["dim"] == 1:
        return 0.05 * np.sin(2 * np.pi * w["x"])
    X, Y = w["x"]
    return 0.05 * np.stack([np.sin(2 * np.pi * (X + Y)), np.cos(2 * np.pi * (X - Y))])


@pytest.mark.parametrize("case", list(CASES))
def test_rhs_parity_walls(case):
    import torch

    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    xd = _xdot(w)
    dU_o, dJ_o = op.rhs(sch, JU_o, J_o, x, xd)
    dU, dJ = torch.empty_like(JU), torch.empty_like(J)
    es.es_rhs(ctx, JU, J, xt, torch.tensor(np.ascontiguousarray(xd), device="cuda"), dU, dJ)
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    scale = np.abs(JU_o).sum() / min(w["dxi"])
    assert np.abs(to_np(dU) - dU_o).sum() / scale < 1e-12
    assert np.abs(to_np(dJ) - dJ_o).sum() / (np.abs(J_o).sum() / min(w["dxi"])) < 1e-12
    assert np.abs(dU_o).sum() > 1e-6 * scale * min(w["dxi"])


@pytest.mark.parametrize("case", list(CASES))
def test_mesh_redistribution_parity_walls(case):
    import torch

    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    sch, mc, JU_o, J_o, x = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    xdot_o, sw_o, gam_o = stepper.redistribute(sch, mc, JU_o, J_o, x, 0.002)
    xdot = torch.empty_like(xt)
    sw, gam = es.es_mesh_redistribute(ctx, JU, J, xt, 0.002, xdot)
    assert sw == sw_o and abs(gam - gam_o) <= 1e-12 * gam_o
    assert np.abs(xdot_o).max() > 0.0
    assert np.abs(to_np(xdot) - xdot_o).max() <= 1e-11 * np.abs(xdot_o).max()


@pytest.mark.parametrize("case", list(CASES))
def test_step_parity_walls(case):
    from paper_2407_05568_gb300 import es
    w = CASES[case]()
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    t = 0.0
    for _ in range(2):
        JU_o, J_o, x_o, t, _ = stepper.step(sch, mc, JU_o, J_o, x_o, t, w["t_end"], w["cfl"])
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, 2, w["t_end"])
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    assert rel_l1(to_np(JU), JU_o) < 2e-12
    assert rel_l1(to_np(J), J_o) < 2e-12
    assert rel_l1(to_np(xt), x_o) < 2e-12
