"""Pins of the oracle's MR-WENO5 reconstruction."""
from fractions import Fraction

import numpy as np

from oracle import weno


def _cell_averages(coefs, centers):
    """Exact unit-cell averages of the polynomial sum_k coefs[k] x^k."""
    out = []
    for c in centers:
        tot = 0.0
        for k, a in enumerate(coefs):
            tot += a * (((c + 0.5) ** (k + 1) - (c - 0.5) ** (k + 1)) / (k + 1))
        out.append(tot)
    return np.array(out)


def test_textbook_interface_weights():
    """The 3- and 5-point interface values are the textbook ones: (-1, 5, 2)/6 and (2, -13, 47, 27, -3)/60."""
    assert weno.interface_weights((-1, 0, 1)) == [Fraction(-1, 6), Fraction(5, 6), Fraction(2, 6)]
    assert weno.interface_weights((-2, -1, 0, 1, 2)) == [Fraction(c, 60) for c in (2, -13, 47, 27, -3)]


def test_jiang_shu_three_point_indicator():
    """beta_2 from the definition equals 13/12 (w_-1 - 2 w_0 + w_1)^2 + 1/4 (w_1 - w_-1)^2."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        w = rng.normal(size=3)
        ref = 13 / 12 * (w[0] - 2 * w[1] + w[2]) ** 2 + 0.25 * (w[2] - w[0]) ** 2
        assert np.isclose(w @ weno._B2 @ w, ref, rtol=1e-13)


def test_linear_limit_is_exact_for_quartics():
    """With the linear weights (eps -> infinity) the result is q_3: exact on degree-4 polynomials."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        c = rng.normal(size=5)
        w = _cell_averages(c, range(-2, 3))
        exact = sum(a * 0.5**k for k, a in enumerate(c))
        assert np.isclose(weno.mr_weno5(w, eps=1e30), exact, rtol=1e-12, atol=1e-12)


def test_constants_exact():
    """A constant sequence is reproduced by every p_l, hence by any weights (up to rounding)."""
    w = np.full((5, 7), 3.25)
    w[:, 3] = -1.5
    out = weno.mr_weno5(w)
    assert np.allclose(out, w[2], rtol=4e-16, atol=0)


def test_design_order_on_smooth_data():
    """Point values of a smooth function, reconstructed at i+1/2, converge at fifth order."""
    errs = []
    for n in (20, 40, 80, 160):
        h = 1.0 / n
        x = np.arange(n) * h
        # w_i are point values of u(x) = sin(2 pi x); the FD-WENO target is the interface
        # value of the flux function whose sliding averages are u: f(x_{i+1/2}) with
        # f = u - h^2/24 u'' + 7 h^4/5760 u'''' - ... ; we compare against the exact primitive form.
        u = np.sin(2 * np.pi * x)
        st = np.stack([np.roll(u, -o) for o in range(-2, 3)])
        rec = weno.mr_weno5(st)
        # exact: the function H with (1/h) int_{x-h/2}^{x+h/2} H = u has H(x+h/2) =
        # sin(2 pi (x + h/2)) * (pi h) / sin(pi h)
        ex = np.sin(2 * np.pi * (x + h / 2)) * (np.pi * h) / np.sin(np.pi * h)
        errs.append(np.abs(rec - ex).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 4.5, (errs, orders)


def test_discontinuity_picks_smooth_stencil():
    """Near a jump the nonlinear weights move to the low-order candidates (no new extremum)."""
    w = np.array([1.0, 1.0, 1.0, 0.0, 0.0])
    r = weno.mr_weno5(w)
    assert 0.0 <= r <= 1.0 + 1e-12


def test_shift_equivariance_on_small_variations():
    """Adding a constant C to the data adds C to the reconstruction: the smoothness indicators
    integrate derivatives, which ignore C, and every candidate reproduces constants.  With a large
    mean and a variation near the indicator regulariser this holds only if the indicators are not
    formed from |w|^2-sized terms."""
    rng = np.random.default_rng(8)
    base = 1e-6 * np.cumsum(rng.standard_normal((5, 400)), axis=0)
    for C in (8.47, -250.0, 3.0e3):
        for g in ((0.005, 0.045, 0.95), (1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0)):
            r0 = weno.mr_weno5(base, g, 1e-12)
            r1 = weno.mr_weno5(base + C, g, 1e-12)
            # the shifted data themselves are rounded to the spacing of C
            tol = 1e-3 * np.abs(base).max() + 64 * np.spacing(abs(C))
            assert np.abs((r1 - C) - r0).max() < tol, (C, g)
