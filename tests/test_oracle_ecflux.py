"""Pins of the oracle's two-point EC flux (Sec. 3.1)."""
import mpmath
import numpy as np
import pytest

from oracle import ecflux, thermo


def _admissible_pairs(g, n, rng, d=2, near=False):
    """Random admissible (rho, v, T) pairs satisfying the condition of Theorem 3.1."""
    out = []
    while len(out) < n:
        rl, rr = rng.uniform(0.2, 2.4, 2)
        Tl, Tr = rng.uniform(0.9, 1.8, 2)
        if near:
            rr = rl * (1 + rng.uniform(-1e-6, 1e-6))
            Tr = Tl * (1 + rng.uniform(-1e-6, 1e-6))
        if g.b > 0:
            ok = all(thermo.admissible(g, np.array(r), np.array(T)) for r, T in ((rl, Tl), (rr, Tr)))
            rm, Tm = 0.5 * (rl + rr), 0.5 * (Tl + Tr)
            ok = ok and (g.R * Tm - 2 * g.a * rm * (1 - g.b * rm) ** 2 > 0)
            if not ok:
                continue
        out.append((rl, rng.uniform(-1, 1, d), Tl, rr, rng.uniform(-1, 1, d), Tr))
    rl = np.array([o[0] for o in out])
    vl = np.array([o[1] for o in out]).T
    Tl = np.array([o[2] for o in out])
    rr = np.array([o[3] for o in out])
    vr = np.array([o[4] for o in out]).T
    Tr = np.array([o[5] for o in out])
    return rl, vl, Tl, rr, vr, Tr


GASES = {"units_a": thermo.gas_units_a(), "units_b": thermo.gas_units_b(), "ideal": thermo.ideal_gas(1.4)}


def test_log_mean_against_multiprecision():
    """{a}^ln = [[a]]/[[ln a]] evaluated in 40-digit arithmetic, including near-equal pairs."""
    mpmath.mp.dps = 40
    rng = np.random.default_rng(0)
    a = rng.uniform(0.1, 3.0, 300)
    b = np.concatenate([rng.uniform(0.1, 3.0, 100), a[100:200] * (1 + rng.uniform(-1e-2, 1e-2, 100)),
                        a[200:] * (1 + rng.uniform(-1e-9, 1e-9, 100))])
    lm = ecflux.log_mean(a, b)
    for x, y, m in zip(a, b, lm):
        X, Y = mpmath.mpf(float(x)), mpmath.mpf(float(y))
        ref = X if X == Y else (X - Y) / (mpmath.log(X) - mpmath.log(Y))
        assert abs(m - float(ref)) <= 4e-16 * float(ref)
    assert ecflux.log_mean(2.0, 2.0) == 2.0


@pytest.mark.parametrize("gname", list(GASES))
def test_consistency(gname):
    """Remark after Theorem 3.1: U~(U, U) = U and F~_j(U, U) = F_j(U)."""
    g = GASES[gname]
    rng = np.random.default_rng(1)
    rl, vl, Tl, _, _, _ = _admissible_pairs(g, 200, rng)
    Ut, Ft = ecflux.ec_flux(g, rl, vl, Tl, rl, vl, Tl)
    U = thermo.prim_to_cons(g, rl, vl, thermo.pressure(g, rl, Tl))
    scale = np.abs(U).max(axis=0)
    assert np.all(np.abs(Ut - U) <= 1e-13 * scale)
    for j in range(2):
        n = np.zeros((2, 1))
        n[j] = 1.0
        F = thermo.flux(g, U, n)
        assert np.all(np.abs(Ft[j] - F) <= 1e-13 * np.abs(F).max(axis=0).clip(min=scale * 1e-3))


@pytest.mark.parametrize("gname", list(GASES))
def test_symmetry(gname):
    """U~ and F~_j are symmetric in (l, r) (Sec. 3.1, after eq. ECfluxMM)."""
    g = GASES[gname]
    rng = np.random.default_rng(2)
    rl, vl, Tl, rr, vr, Tr = _admissible_pairs(g, 200, rng)
    a = ecflux.ec_flux(g, rl, vl, Tl, rr, vr, Tr)
    b = ecflux.ec_flux(g, rr, vr, Tr, rl, vl, Tl)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-13, atol=0)


@pytest.mark.parametrize("gname", list(GASES))
def test_tadmor_condition(gname):
    """eq. ECCondition_comp: [[V]].U~ = [[phi]] and [[V]].F~_j = [[psi_j]] to 1e-13 relative."""
    g = GASES[gname]
    rng = np.random.default_rng(4)
    rl, vl, Tl, rr, vr, Tr = _admissible_pairs(g, 4000, rng)
    Ul = thermo.prim_to_cons(g, rl, vl, thermo.pressure(g, rl, Tl))
    Ur = thermo.prim_to_cons(g, rr, vr, thermo.pressure(g, rr, Tr))
    dV = thermo.entropy_variables(g, Ur) - thermo.entropy_variables(g, Ul)
    Ut, Ft = ecflux.ec_flux(g, rl, vl, Tl, rr, vr, Tr)
    lhs = np.sum(dV * Ut, axis=0)
    rhs = thermo.potential(g, Ur) - thermo.potential(g, Ul)
    scale = np.sum(np.abs(dV * Ut), axis=0) + np.abs(rhs) + 1e-300
    assert np.max(np.abs(lhs - rhs) / scale) < 1e-13
    for j in range(2):
        lhs = np.sum(dV * Ft[j], axis=0)
        rhs = thermo.flux_potential(g, Ur, j) - thermo.flux_potential(g, Ul, j)
        scale = np.sum(np.abs(dV * Ft[j]), axis=0) + np.abs(rhs) + 1e-300
        assert np.max(np.abs(lhs - rhs) / scale) < 1e-13


def _mp_entropy_side(g, rho, v, T):
    """V, phi, psi in 40-digit arithmetic from primitive inputs (test harness for tiny jumps)."""
    rho, T = mpmath.mpf(float(rho)), mpmath.mpf(float(T))
    v = [mpmath.mpf(float(x)) for x in v]
    a, b, R, cv = (mpmath.mpf(float(t)) for t in (g.a, g.b, g.R, g.cv))
    s = cv * mpmath.log(T) + R * mpmath.log((1 - b * rho) / rho)
    V1 = cv - s - 2 * a * rho / T + R / (1 - b * rho) - sum(x * x for x in v) / (2 * T)
    V = [V1] + [x / T for x in v] + [-1 / T]
    p = rho * R * T / (1 - b * rho) - a * rho**2
    return V, p / T, [p * x / T for x in v]


@pytest.mark.parametrize("gname", list(GASES))
def test_tadmor_condition_near_equal_states(gname):
    """Same condition for states 1e-6 apart; the jumps of V are taken in 40-digit arithmetic."""
    mpmath.mp.dps = 40
    g = GASES[gname]
    rng = np.random.default_rng(5)
    rl, vl, Tl, rr, vr, Tr = _admissible_pairs(g, 150, rng, near=True)
    vr = vl * (1 + rng.uniform(-1e-6, 1e-6, vl.shape))
    Ut, Ft = ecflux.ec_flux(g, rl, vl, Tl, rr, vr, Tr)
    for i in range(rl.size):
        Vl, phl, psl = _mp_entropy_side(g, rl[i], vl[:, i], Tl[i])
        Vr, phr, psr = _mp_entropy_side(g, rr[i], vr[:, i], Tr[i])
        dV = [x - y for x, y in zip(Vr, Vl)]
        for vec, rhs in [(Ut[:, i], phr - phl)] + [(Ft[j][:, i], psr[j] - psl[j]) for j in range(2)]:
            terms = [dv * mpmath.mpf(float(u)) for dv, u in zip(dV, vec)]
            err = abs(sum(terms) - rhs)
            scale = sum(abs(t) for t in terms) + abs(rhs)
            assert float(err / scale) < 1e-13


def test_matches_paper_reduced_formula():
    """The general-unit restatement equals the paper's printed reduced-unit U~, F~_1 (1D)."""
    g = thermo.gas_units_b()
    rng = np.random.default_rng(7)
    rl, vl, Tl, rr, vr, Tr = _admissible_pairs(g, 500, rng, d=1)
    Ut, Ft = ecflux.ec_flux(g, rl, vl, Tl, rr, vr, Tr)
    Up, Fp = ecflux.ec_flux_units_b_1d(0.0125, (rl, vl[0], Tl), (rr, vr[0], Tr))
    assert np.allclose(Ut, Up, rtol=1e-13, atol=1e-13)
    assert np.allclose(Ft[0], Fp, rtol=1e-12, atol=1e-12)


def test_theorem_3_1_determinant_positive():
    """Theorem 3.1: D > 0 whenever 4{T} - {rho}(3 - {rho})^2 > 0 (reduced units)."""
    g = thermo.gas_units_a()
    rng = np.random.default_rng(8)
    rl, vl, Tl, rr, vr, Tr = _admissible_pairs(g, 5000, rng)
    D = ecflux.ec_determinant(g, rl, Tl, rr, Tr)
    assert np.all(D > 0)


def test_ideal_gas_density_mean():
    """a = b = 0: U~_1 reduces to the logarithmic mean of rho (the Ismail-Roe density flux)."""
    g = thermo.ideal_gas(1.4)
    rng = np.random.default_rng(9)
    rl, vl, Tl, rr, vr, Tr = _admissible_pairs(g, 100, rng)
    Ut, _ = ecflux.ec_flux(g, rl, vl, Tl, rr, vr, Tr)
    assert np.allclose(Ut[0], ecflux.log_mean(rl, rr), rtol=1e-14)
