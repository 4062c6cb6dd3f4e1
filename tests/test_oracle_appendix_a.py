"""Appendix A's alternative parameter vectors as negative tests: their linear systems can be singular where the
system of Sec. 3.1 is not.

For three other vectors z, App. A writes [[V]] = M [[z]] (1D, the paper's reduced units) and prints det M.  Pins:
  * each printed system reproduces the jump of the entropy variables (the oracle's V in the reduced units), so the
    transcription is the paper's system;
  * the printed determinants equal det M for the second and third vectors; for the first, det M is
    3 {1/T} ((B{z2} - A{z1})/{3 z1 z2 - 1}^ln + B{z2} - A{z1} + (3/4) B), where the paper prints 3/4 without the
    factor B = {z1}^2 (a garbled point; the expansion of det M is exact, checked symbolically and numerically);
  * for each vector there are admissible pairs of states at which its determinant vanishes while D of Theorem 3.1
    stays positive, and there the EC flux of Sec. 3.1 exists and satisfies Tadmor's condition.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import appendix_a as aa
from oracle import ecflux, thermo

DELTA = 0.0125
VECTORS = {1: aa.vector_1, 2: aa.vector_2, 3: aa.vector_3}


def _admissible(rho, T):
    """eq. coefflimit in the reduced units: 0 < rho < 3, T > 27/32, 4T - rho (3 - rho)^2 > 0."""
    return 0.0 < rho < 3.0 and T > 27.0 / 32.0 and 4.0 * T - rho * (3.0 - rho) ** 2 > 0.0


def _V(g, rho, v, T):
    U = thermo.prim_to_cons(g, np.array([rho]), np.array([[v]]), thermo.pressure(g, np.array([rho]), np.array([T])))
    return thermo.entropy_variables(g, U)[:, 0]


def _random_pairs(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        rl, rr = rng.uniform(0.05, 2.9, 2)
        Tl, Tr = rng.uniform(0.86, 1.8, 2)
        vl, vr = rng.uniform(-0.6, 0.6, 2)
        if _admissible(rl, Tl) and _admissible(rr, Tr):
            out.append(((rl, vl, Tl), (rr, vr, Tr)))
    return out


@pytest.mark.parametrize("k", [1, 2, 3])
def test_printed_system_reproduces_the_jump_of_v(k):
    g = thermo.gas_units_b(DELTA)
    for l, r in _random_pairs(200, k):
        M, zl, zr, _ = VECTORS[k](l, r, DELTA)
        dV = _V(g, *r) - _V(g, *l)
        assert np.abs(M @ (zr - zl) - dV).max() <= 1e-11 * np.abs(dV).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_determinant(k):
    for l, r in _random_pairs(200, 10 + k):
        M, _, _, det = VECTORS[k](l, r, DELTA)
        assert abs(np.linalg.det(M) - det) <= 1e-10 * max(abs(det), np.abs(M).max() ** 3 * 1e-6)


def test_first_determinant_as_printed_differs():
    """Without the factor {z1}^2 on 3/4 (as printed) the first determinant is another function: at equal states it
    would vanish at rho = 4/T for any T > 4/3, while det M there is 9/(4 rho T^3) (rho (3 - rho)^2 - 4T) < 0."""
    T, rho = 1.5, 4.0 / 1.5
    M, zl, zr, det = aa.vector_1((rho, 0.0, T), (rho, 0.0, T), DELTA)
    z1, z2 = zl[0], zl[1]
    printed = 3.0 / T * (-(z1 * z2) * z1 / (rho / (3.0 - rho)) - z1 * z2 * z1 + 0.75)
    assert abs(printed) < 1e-12
    assert det == pytest.approx(9.0 / (4.0 * rho * T**3) * (rho * (3.0 - rho) ** 2 - 4.0 * T), rel=1e-12)
    assert np.linalg.det(M) == pytest.approx(det, rel=1e-12) and det < -0.1


# (left state (rho, T), right temperature, bracket of the right density) with the right density moving
SINGULAR = {1: ((1.4589, 0.9505), 0.9433, (0.5404, 0.5493)),
            2: ((0.8905, 1.0243), 0.8597, (1.5719, 1.5819)),
            3: ((0.8905, 1.0243), 0.8597, (1.5719, 1.5819))}


@pytest.mark.parametrize("k", [1, 2, 3])
def test_alternative_singular_where_section_3_1_is_not(k):
    (rl, Tl), Tr, (a, b) = SINGULAR[k]
    f = VECTORS[k]

    def det(rr):
        return np.linalg.det(f((rl, 0.3, Tl), (rr, -0.2, Tr), DELTA)[0])

    assert det(a) * det(b) < 0.0
    for rr in np.linspace(a, b, 21):
        assert _admissible(rl, Tl) and _admissible(rr, Tr)
        assert aa.theorem_3_1_D((rl, 0.0, Tl), (rr, 0.0, Tr)) > 1e-3
    root = brentq(det, a, b, xtol=1e-15)
    M = f((rl, 0.3, Tl), (root, -0.2, Tr), DELTA)[0]
    assert np.linalg.cond(M) > 1e9
    # the paper's own system is uniquely solvable there: its EC flux satisfies Tadmor's condition
    g = thermo.gas_units_b(DELTA)
    Ut, Ft = ecflux.ec_flux(g, np.array([rl]), np.array([[0.3]]), np.array([Tl]),
                            np.array([root]), np.array([[-0.2]]), np.array([Tr]))
    Ul = thermo.prim_to_cons(g, np.array([rl]), np.array([[0.3]]), thermo.pressure(g, np.array([rl]), np.array([Tl])))
    Ur = thermo.prim_to_cons(g, np.array([root]), np.array([[-0.2]]),
                             thermo.pressure(g, np.array([root]), np.array([Tr])))
    dV = thermo.entropy_variables(g, Ur) - thermo.entropy_variables(g, Ul)
    dphi = thermo.potential(g, Ur) - thermo.potential(g, Ul)
    dpsi = thermo.flux_potential(g, Ur, 0) - thermo.flux_potential(g, Ul, 0)
    assert np.all(np.isfinite(Ut)) and np.all(np.isfinite(Ft))
    assert abs(np.sum(dV * Ut) - dphi[0]) <= 1e-12 * np.sum(np.abs(dV * Ut))
    assert abs(np.sum(dV * Ft[0]) - dpsi[0]) <= 1e-12 * np.sum(np.abs(dV * Ft[0]))
