"""Pins of the wall and symmetry-plane boundaries (a reading: the paper does not specify its
boundary conditions; Example 5.7's octant needs symmetry planes through the sphere's centre).

A symmetry plane at the low end of a direction must reproduce the mirror-symmetric solution of the
full domain: the state mirrored about the boundary node with the normal momentum negated.  So the
half (1D), quarter (2D) and octant (3D) problems are checked against the full problems with
outflow boundaries, for the right-hand side and for whole moving-mesh steps.  A wall at both ends
keeps a gas at rest at rest.
"""
import numpy as np
import pytest

from oracle import stepper, thermo
from oracle import operator as op
from paper_2407_05568_gb300 import workloads as wl


def _axis(n, lo, hi):
    return wl.uniform_nodes(n, lo, hi, False)


def _state(g, xs):
    """Mirror-symmetric supercritical state: rho, p even in every coordinate, v_k odd in x_k."""
    r2 = sum(x**2 for x in xs)
    inside = r2 < 0.17                      # a radius between nodes: rounding decides no node
    rho = np.where(inside, 1.2, 0.6) + 0.05 * np.exp(-10 * r2)
    p = np.where(inside, 1.8, 1.0)
    v = np.stack([0.2 * x * np.exp(-r2) for x in xs])
    return thermo.prim_to_cons(g, rho, v, p)


def _setup(dim, n, half):
    g = thermo.gas_units_a()
    a, d = _axis(n, 0.0, 1.0)
    if half:
        bc = (op.SYMMETRY_LO,) * dim
    else:
        a = np.concatenate([-a[:0:-1], a])          # mirrored nodes are exact negatives
        bc = (op.OUTFLOW,) * dim
    grids = np.meshgrid(*([a] * dim), indexing="ij")[::-1]      # x_1 along the last axis
    x = np.stack(grids)
    sch = op.Scheme(gas=g, dim=dim, bc=bc, dxi=(d,) * dim, period=(2.0,) * dim)
    J = op.node_jacobian(sch, x)
    U = _state(g, list(x))
    return sch, U * J, J, x


def _part(a, dim, n, lead=1):
    """The x_k >= 0 part of a full-domain field (the last `dim` axes)."""
    sl = (slice(None),) * lead + (slice(n - 1, None),) * dim
    return a[sl]


@pytest.mark.parametrize("dim,n", [(1, 24), (2, 14), (3, 9)])
def test_symmetry_plane_reproduces_the_full_domain_rhs(dim, n):
    sch_h, JU_h, J_h, x_h = _setup(dim, n, True)
    sch_f, JU_f, J_f, x_f = _setup(dim, n, False)
    assert np.allclose(_part(x_f, dim, n), x_h, rtol=0, atol=1e-15)
    dU_h, dJ_h = op.rhs(sch_h, JU_h, J_h, x_h, np.zeros_like(x_h))
    dU_f, dJ_f = op.rhs(sch_f, JU_f, J_f, x_f, np.zeros_like(x_f))
    scale = np.abs(dU_f).max()
    assert scale > 0
    assert np.abs(dU_h - _part(dU_f, dim, n)).max() < 1e-11 * scale


@pytest.mark.parametrize("dim,n,steps", [(1, 40, 3), (2, 16, 1)])
def test_symmetry_plane_reproduces_full_domain_moving_mesh_steps(dim, n, steps):
    """Whole steps with the moving mesh: the full domain's centre nodes stay on the planes by
    symmetry, the half domain pins their normal coordinate; time steps, meshes and states agree."""
    mc = stepper.MeshControl(moving=True, monitor="vdw", alphas=(1200.0, 1200.0, 1200.0), kappa=2,
                             filter_passes=3, sweeps=5)
    sch_h, JU_h, J_h, x_h = _setup(dim, n, True)
    sch_f, JU_f, J_f, x_f = _setup(dim, n, False)
    t_h = t_f = 0.0
    for _ in range(steps):
        JU_h, J_h, x_h, t_h, _ = stepper.step(sch_h, mc, JU_h, J_h, x_h, t_h, 1.0, 0.4)
        JU_f, J_f, x_f, t_f, _ = stepper.step(sch_f, mc, JU_f, J_f, x_f, t_f, 1.0, 0.4)
    assert abs(t_h - t_f) <= 1e-13 * t_f
    assert np.abs(x_h - _part(x_f, dim, n)).max() < 1e-13
    assert np.abs(JU_h - _part(JU_f, dim, n)).max() < 1e-11 * np.abs(JU_f).max()


@pytest.mark.parametrize("dim", [1, 2])
def test_walls_keep_a_gas_at_rest(dim):
    n = 20
    g = thermo.gas_units_a()
    a, d = _axis(n, 0.0, 1.0)
    x = np.stack(np.meshgrid(*([a] * dim), indexing="ij")[::-1])
    sch = op.Scheme(gas=g, dim=dim, bc=(op.REFLECT,) * dim, dxi=(d,) * dim, period=(1.0,) * dim)
    J = op.node_jacobian(sch, x)
    U = thermo.prim_to_cons(g, np.full(x.shape[1:], 0.8), np.zeros(x.shape), np.full(x.shape[1:], 1.1))
    dU, dJ = op.rhs(sch, U * J, J, x, np.zeros_like(x))
    assert np.abs(dU).max() < 1e-12 * np.abs(U).max() / d


def test_wall_mirrors_the_normal_momentum_only():
    """pad_state at a wall: density and energy mirror, the normal momentum changes sign, the
    tangential momentum mirrors."""
    U = np.arange(1.0, 1.0 + 4 * 6 * 5).reshape(4, 6, 5)        # (rho, m1, m2, E) on n2 = 6, n1 = 5
    P = op.pad_state(U, 3, 0, 2, op.REFLECT)                        # direction xi_1 (last axis)
    assert np.array_equal(P[0][:, 2], U[0][:, 1]) and np.array_equal(P[0][:, 0], U[0][:, 3])
    assert np.array_equal(P[1][:, 2], -U[1][:, 1]) and np.array_equal(P[1][:, -1], -U[1][:, -4])
    assert np.array_equal(P[2][:, 2], U[2][:, 1]) and np.array_equal(P[3][:, -3], U[3][:, -2])
    Q = op.pad_state(U, 3, 1, 2, op.SYMMETRY_LO)                    # direction xi_2: mirror low, copy high
    assert np.array_equal(Q[2][2], -U[2][1]) and np.array_equal(Q[2][-1], U[2][-1])
