"""Pins of the oracle's warm-start parts: the conv net (forward, backward, Adam,
bf16 rounding) and the guarded mesh solve, against library routines, finite
differences, closed forms and invariants."""
import os

import numpy as np
import pytest

from oracle import convnet, mesh, warmstart
from oracle import operator as op
from oracle import stepper, thermo
from paper_2407_05568_gb300 import workloads as wl

from sides import oracle_setup

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table_5_1.txt")


def test_bf16_round_matches_torch():
    """Round-to-nearest-even bf16 against torch's own float32 -> bfloat16 conversion."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-8, 8, 20000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.0078125, 1.005859375, 3.0e38, -1e-40],
                                 dtype=np.float32)])
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(convnet.bf16_round(a), ref)


def test_bf16_round_ties_to_even():
    """1 + 2^-8 lies halfway between bf16 neighbours 1 and 1 + 2^-7: it rounds to the even one (1)."""
    assert convnet.bf16_round(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert convnet.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6
    assert convnet.bf16_round(np.float32(1.0 + 2.0 ** -7)) == 1.0 + 2.0 ** -7


def test_conv3x3_matches_scipy_correlate():
    """z[co] = b[co] + sum_ci correlate2d(a[ci], w[co, ci], 'same', zero fill)."""
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 3, 7, 9))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    z = convnet.conv3x3(a, w, b)
    for n in range(2):
        for co in range(4):
            ref = b[co] + sum(signal.correlate2d(a[n, ci], w[co, ci], mode="same", boundary="fill", fillvalue=0.0)
                              for ci in range(3))
            assert np.allclose(z[n, co], ref, rtol=1e-13, atol=1e-13)


def test_conv3x3_delta_kernel_shifts():
    """A kernel with a single 1 at (dy, dx) returns the input shifted by (dy - 1, dx - 1), zero outside."""
    rng = np.random.default_rng(2)
    a = rng.standard_normal((1, 1, 6, 5))
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 2, 0] = 1.0                     # z(y, x) = a(y + 1, x - 1)
    z = convnet.conv3x3(a, w)[0, 0]
    assert np.array_equal(z[:-1, 1:], a[0, 0, 1:, :-1])
    assert np.all(z[-1, :] == 0.0) and np.all(z[:, 0] == 0.0)


def _net(rng, cin=4, hidden=3, cout=2, layers=3):
    chans = [cin] + [hidden] * (layers - 1) + [cout]
    ws = [rng.standard_normal((chans[l + 1], chans[l], 3, 3)) * 0.4 for l in range(layers)]
    bs = [rng.standard_normal(chans[l + 1]) * 0.1 for l in range(layers)]
    return ws, bs


def test_backward_matches_finite_differences():
    """dL/dw, dL/db of the MSE through tanh layers against central differences (float64)."""
    rng = np.random.default_rng(3)
    ws, bs = _net(rng)
    a0 = rng.standard_normal((2, 4, 5, 6))
    tgt = rng.standard_normal((2, 2, 5, 6))

    def loss(ws_, bs_):
        return convnet.mse(convnet.forward(ws_, bs_, a0)[-1], tgt)[0]

    acts = convnet.forward(ws, bs, a0)
    _, g = convnet.mse(acts[-1], tgt)
    gws, gbs = convnet.backward(ws, acts, g)
    h = 1e-6
    for l in range(len(ws)):
        for idx in [(0, 0, 0, 0), (1, 2, 1, 2), (-1, -1, 2, 1)]:
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[l][idx] += h
            wm[l][idx] -= h
            fd = (loss(wp, bs) - loss(wm, bs)) / (2 * h)
            assert abs(fd - gws[l][idx]) <= 1e-7 * max(1.0, abs(fd)), (l, idx, fd, gws[l][idx])
        for c in range(bs[l].size):
            bp = [b.copy() for b in bs]
            bm = [b.copy() for b in bs]
            bp[l][c] += h
            bm[l][c] -= h
            fd = (loss(ws, bp) - loss(ws, bm)) / (2 * h)
            assert abs(fd - gbs[l][c]) <= 1e-7 * max(1.0, abs(fd))


def test_input_gradient_matches_finite_differences():
    """dL/da of one layer (the input-gradient correlation with the flipped kernel)."""
    rng = np.random.default_rng(4)
    a = rng.standard_normal((1, 3, 4, 5))
    w = rng.standard_normal((2, 3, 3, 3))
    r = rng.standard_normal((1, 2, 4, 5))

    def L(a_):
        return float(np.sum(r * convnet.conv3x3(a_, w)))

    _, _, ga = convnet.conv3x3_backward(a, w, r)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 2, 3), (0, 2, 3, 4), (0, 0, 3, 0)]:
        ap = a.copy()
        am = a.copy()
        ap[idx] += h
        am[idx] -= h
        assert abs((L(ap) - L(am)) / (2 * h) - ga[idx]) < 1e-7


def test_adam_first_step_closed_form():
    """With m = v = 0, the bias-corrected first Adam step is -lr g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 2.0, 3.0, 4.0])
    t1, m, v = convnet.adam(th, g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-8)
    assert np.allclose(t1, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_descends_quadratic():
    """Adam on f = |theta|^2 / 2 from theta = 1 approaches the minimum."""
    th = np.ones(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for k in range(1, 2001):
        th, m, v = convnet.adam(th, th, m, v, k, lr=0.01)
    assert np.abs(th).max() < 1e-2


# ----------------------------------------------------------------- guarded mesh solve
def _riemann(n=24, sweeps=12, eps=0.0):
    w = wl.riemann_2d(n, seed=5)
    w["mesh"] = dict(w["mesh"], sweeps=sweeps, eps=eps)
    return oracle_setup(w)


def test_solve_without_start_is_plain_jacobi():
    sch, mc, JU, J, x = _riemann()
    om, _ = warmstart.filtered_monitor(sch, mc, JU, J)
    xp, kp = mesh.jacobi(sch, x, om, mc.sweeps, mc.eps)
    xs, ks, picked = warmstart.solve(sch, mc, JU, J, x)
    assert np.array_equal(xs, xp) and ks == kp and picked == 0


def test_filtered_monitor_matches_redistribute():
    """The monitor feeding the features is the one the plain redistribution uses: with a
    zero-change limiter the plain step's displacement equals the plain Jacobi iterate's."""
    sch, mc, JU, J, x = _riemann(sweeps=5)
    xd, sw, gam = stepper.redistribute(sch, mc, JU, J, x, 1.0)
    xs, ks, _ = warmstart.solve(sch, mc, JU, J, x)
    assert ks == sw
    assert np.allclose(xd, gam * (xs - x), rtol=0, atol=1e-15)


def test_guarded_start_from_plain_iterate_continues_it():
    """Starting from the plain iterate x^[3], mu sweeps give the plain x^[3 + mu] exactly."""
    sch, mc, JU, J, x = _riemann(sweeps=6)
    om, _ = warmstart.filtered_monitor(sch, mc, JU, J)
    x3, _ = mesh.jacobi(sch, x, om, 3)
    x9, _ = mesh.jacobi(sch, x, om, 9)
    xs, ks, picked = warmstart.solve(sch, mc, JU, J, x, x_start=x3)
    assert picked == 1 and ks == 6
    assert np.array_equal(xs, x9)


def test_guard_rejects_a_bad_start():
    """A start with large random displacements loses the guard: the plain iterate results."""
    sch, mc, JU, J, x = _riemann(sweeps=6)
    rng = np.random.default_rng(7)
    bad = warmstart.warm_start(sch, x, rng.standard_normal(x.shape) * 0.4)
    xs, ks, picked = warmstart.solve(sch, mc, JU, J, x, x_start=bad)
    xp, kp, _ = warmstart.solve(sch, mc, JU, J, x)
    assert picked == 0 and ks == kp
    assert np.array_equal(xs, xp)


def test_tolerance_stops_the_warm_path_early():
    """With eps set, a start at the plain iterate's end needs only the guarded sweep."""
    eps = 0.02 / 23                         # 2% of a cell
    sch, mc, JU, J, x = _riemann(sweeps=400, eps=eps)
    xp, kp, _ = warmstart.solve(sch, mc, JU, J, x)
    assert 10 < kp < 400
    xs, ks, picked = warmstart.solve(sch, mc, JU, J, x, x_start=xp)
    assert picked == 1 and ks == 1
    assert np.abs(xs - xp).max() < eps


def test_warm_start_keeps_fixed_nodes_and_drops_nonfinite():
    sch, mc, JU, J, x = _riemann()
    out = np.full(x.shape, 0.25)
    out[0, 5, 5] = np.nan
    xs = warmstart.warm_start(sch, x, out)
    fixed = mesh._fixed_mask(x.shape[1:], 2, sch.bc)          # per component (outflow: all of them)
    for c in range(2):
        assert np.array_equal(xs[c][fixed[c]], x[c][fixed[c]])
    assert xs[0, 5, 5] == x[0, 5, 5]
    inner = ~fixed[0]
    inner[5, 5] = False
    assert np.allclose((xs[0] - x[0])[inner], 0.25 * sch.dxi[0], rtol=1e-12)


def _table():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, side, rho, v, p, G = line.split()
            rows.append((float(rho), float(v), float(p), float(G)))
    return rows


def test_features_on_uniform_states():
    """A constant state on the Cartesian mesh: omega = 1 (ln omega = 0), zero displacement,
    and the G feature equals G/(1+|G|) of the value Table 5.1 prints for that state."""
    g = thermo.gas_units_a()
    n = 12
    for rho, v, p, G_printed in _table():
        sch = op.Scheme(gas=g, dim=2, bc=("outflow", "outflow"), dxi=(1 / (n - 1), 1 / (n - 1)), period=(1.0, 1.0))
        mc = stepper.MeshControl(moving=True)
        X, Y = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
        x = np.stack([X, Y])
        J = op.node_jacobian(sch, x)
        JU = thermo.prim_to_cons(g, np.full((n, n), rho), np.zeros((2, n, n)), np.full((n, n), p)) * J
        f = warmstart.features(sch, mc, JU, J, x)
        assert np.abs(f[0]).max() == 0.0
        assert np.abs(f[2:]).max() < 1e-12
        assert np.abs(f[1] - G_printed / (1 + abs(G_printed))).max() < 1.5e-3


def test_guard_ratio_admits_a_larger_first_residual():
    """Grid-scale noise of 0.1 cells on a good start doubles its first residual: refused at
    ratio 1, kept at ratio 4, and then continued exactly like the plain iteration from it."""
    sch, mc, JU, J, x = _riemann(sweeps=6)
    om, _ = warmstart.filtered_monitor(sch, mc, JU, J)
    x12, _ = mesh.jacobi(sch, x, om, 12)
    rng = np.random.default_rng(12)
    xs = warmstart.warm_start(sch, x12, rng.standard_normal(x.shape) * 0.1)
    _, _, p1 = warmstart.solve(sch, mc, JU, J, x, xs, guard_ratio=1.0)
    x4, k4, p4 = warmstart.solve(sch, mc, JU, J, x, xs, guard_ratio=4.0)
    ref, _ = mesh.jacobi(sch, xs, om, 6)
    assert (p1, p4, k4) == (0, 1, 6)
    assert np.array_equal(x4, ref)


def test_forward_bf16_inputs_rounds_each_layer_input():
    """With bf16_inputs the first layer sees the bf16-rounded features (a value between two bf16
    neighbours moves to one of them) and the rest of the definition is unchanged."""
    rng = np.random.default_rng(13)
    ws, bs = _net(rng, hidden=3, layers=2)
    a0 = (1.0 + 2.0 ** -9) * np.ones((1, 4, 3, 3))          # halfway-below: rounds to 1.0
    plain = convnet.forward(ws, bs, a0)
    rounded = convnet.forward(ws, bs, a0, bf16_inputs=True)
    ref = convnet.forward(ws, bs, np.ones((1, 4, 3, 3)))
    assert np.array_equal(rounded[1], convnet.forward(ws, bs, convnet.bf16_round(a0))[1])
    assert np.array_equal(rounded[1], ref[1])
    assert not np.array_equal(plain[1], ref[1])
