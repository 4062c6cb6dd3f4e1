"""Pins of the oracle's operator, mesh redistribution and time stepping (Sec. 3 - Sec. 5)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import mesh, stepper, thermo
from oracle import operator as op
from paper_2407_05568_gb300 import workloads as wl


def _scheme(w, dissipation=True):
    g = thermo.Gas(**w["gas"])
    return op.Scheme(gas=g, dim=w["dim"], bc=w["bc"], dxi=w["dxi"], period=w["period"],
                     dissipation=dissipation)


def _wavy_mesh(X, Y, amp=0.01):
    """A smooth periodic perturbation of the unit-square mesh (keeps x(X+1,Y) = x + 1)."""
    return np.stack([X + amp * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y),
                     Y + amp * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)])


def _smooth_state(g, X, Y):
    rho = 0.6 + 0.2 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    v = np.stack([0.3 + 0.1 * np.cos(2 * np.pi * Y), -0.2 + 0.1 * np.sin(2 * np.pi * X)])
    p = 1.0 + 0.1 * np.sin(2 * np.pi * Y)
    return thermo.prim_to_cons(g, rho, v, p)


# --------------------------------------------------------------- coefficients

def test_alphas_exact():
    """Sec. 3.1: the alpha_{w,m} conditions hold exactly; w = 3 gives (3/2, -3/10, 1/30)."""
    assert op.ec_alphas(3) == [Fraction(3, 2), Fraction(-3, 10), Fraction(1, 30)]
    assert op.ec_alphas(2) == [Fraction(4, 3), Fraction(-1, 6)]
    for w in (1, 2, 3, 4):
        al = op.ec_alphas(w)
        assert sum(m * a for m, a in enumerate(al, 1)) == 1
        for s in range(2, w + 1):
            assert sum(Fraction(m) ** (2 * s - 1) * a for m, a in enumerate(al, 1)) == 0


def test_central_difference_exact_on_polynomials():
    """delta_k with 2w = 6 differentiates polynomials of degree <= 6 exactly."""
    x = np.arange(-3, 4, dtype=np.float64) * 0.37
    for deg in range(7):
        d = op.central_difference(x**deg, 0, 3)[0] / 0.37
        assert abs(d - (deg * 0.0**(deg - 1) if deg else 0.0)) < 1e-12


# ------------------------------------------------------------------ geometry

@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_discrete_scl(bc):
    """eq. SCL_dis holds to round-off: the metric fluxes of eq. GCL_flux telescope to
    delta_1[delta_2 x] - delta_2[delta_1 x] = 0."""
    w = wl.sine_2d(20)
    w["bc"] = (bc, bc)
    sch = _scheme(w)
    X, Y = w["x"]
    x = _wavy_mesh(X, Y, 0.02)
    zero = np.zeros_like(x)
    g = op.thermo.Gas(**w["gas"])
    U = thermo.prim_to_cons(g, np.full_like(X, 0.8), np.stack([0 * X, 0 * X]), np.full_like(X, 1.0))
    J = op.node_jacobian(sch, x)
    # with v = 0 and constant p, F_j(U) = (0, p e_j, 0): the momentum RHS is -p * SCL residual
    dU, dJ = op.rhs(op.Scheme(gas=g, dim=2, bc=sch.bc, dxi=sch.dxi, period=sch.period,
                              dissipation=False), U * J, J, x, zero)
    assert np.abs(dU[1:3]).max() < 1e-12 * (1.0 / sch.dxi[0])
    assert np.abs(dJ).max() == 0.0


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_free_stream_moving_mesh(bc):
    """Remark after eq. HOstable: a constant state stays constant on a moving mesh,
    d(JU)/dt = U dJ/dt to round-off (relative to the flux scale F/dxi)."""
    w = wl.sine_2d(24)
    w["bc"] = (bc, bc)
    sch = _scheme(w)
    g = sch.gas
    X, Y = w["x"]
    x = _wavy_mesh(X, Y)
    J = op.node_jacobian(sch, x)
    U0 = thermo.prim_to_cons(g, np.full_like(X, 0.8), np.stack([0.3 + 0 * X, -0.2 + 0 * X]),
                             np.full_like(X, 1.1))
    xdot = 0.05 * np.stack([np.sin(2 * np.pi * (X + Y)), np.cos(2 * np.pi * (X - Y))])
    if bc == "outflow":
        xdot[:, [0, -1], :] = 0.0
        xdot[:, :, [0, -1]] = 0.0
    dU, dJ = op.rhs(sch, U0 * J, J, x, xdot)
    scale = np.abs(U0).max() / sch.dxi[0]
    assert np.abs(dU - U0 * dJ).max() < 1e-12 * scale
    assert np.abs(dJ).max() > 1e-3


def test_free_stream_over_steps():
    """Several full SSP-RK3 steps with a moving mesh keep a constant state constant."""
    w = wl.sine_2d(16)
    sch = _scheme(w)
    g = sch.gas
    X, Y = w["x"]
    x = _wavy_mesh(X, Y)
    J = op.node_jacobian(sch, x)
    U0 = thermo.prim_to_cons(g, np.full_like(X, 0.8), np.stack([0.3 + 0 * X, -0.2 + 0 * X]),
                             np.full_like(X, 1.1))
    JU = U0 * J
    xdot = 0.05 * np.stack([np.sin(2 * np.pi * (X + Y)), np.cos(2 * np.pi * (X - Y))])
    dt = 0.2 * sch.dxi[0]
    for _ in range(5):
        JU1, J1 = stepper.rk_stage(sch, 0, dt, JU, J, JU, J, x, xdot)
        JU2, J2 = stepper.rk_stage(sch, 1, dt, JU, J, JU1, J1, x, xdot)
        JU, J = stepper.rk_stage(sch, 2, dt, JU, J, JU2, J2, x, xdot)
        x = x + dt * xdot
    assert np.abs(JU / J - U0).max() < 1e-12 * np.abs(U0).max()


# ------------------------------------------------------------------ entropy

@pytest.mark.parametrize("moving", [False, True])
def test_ec_scheme_conserves_entropy_2d(moving):
    """Sec. 3.1: with the EC flux alone the total entropy rate vanishes on periodic data."""
    w = wl.sine_2d(20)
    sch = _scheme(w, dissipation=False)
    X, Y = w["x"]
    x = _wavy_mesh(X, Y)
    J = op.node_jacobian(sch, x)
    U = _smooth_state(sch.gas, X, Y)
    xdot = (0.05 * np.stack([np.sin(2 * np.pi * (X + Y)), np.cos(2 * np.pi * (X - Y))])
            if moving else np.zeros_like(x))
    dU, dJ = op.rhs(sch, U * J, J, x, xdot)
    V = thermo.entropy_variables(sch.gas, U)
    phi = thermo.potential(sch.gas, U)
    terms = np.sum(V * dU, axis=0) - phi * dJ
    assert abs(terms.sum()) < 1e-13 * np.abs(terms).sum() * 10


def test_ec_scheme_conserves_entropy_1d_moving():
    w = wl.sine_1d(64)
    sch = _scheme(w, dissipation=False)
    xi = w["x"][0]
    x = (xi + 0.02 * np.sin(2 * np.pi * xi))[None]
    J = op.node_jacobian(sch, x)
    rng = np.random.default_rng(0)
    rho = 0.5 + 0.3 * rng.uniform(size=64)        # rough data: the identity is algebraic
    U = thermo.prim_to_cons(sch.gas, rho, rng.uniform(-0.5, 0.5, (1, 64)), 1.0 + 0.2 * rng.uniform(size=64))
    xdot = 0.1 * np.cos(2 * np.pi * xi)[None]
    dU, dJ = op.rhs(sch, U * J, J, x, xdot)
    V = thermo.entropy_variables(sch.gas, U)
    terms = np.sum(V * dU, axis=0) - thermo.potential(sch.gas, U) * dJ
    assert abs(terms.sum()) < 1e-13 * np.abs(terms).sum() * 10


@pytest.mark.parametrize("dim", [1, 2])
def test_es_scheme_produces_entropy(dim):
    """Sec. 3.3: the ES flux dissipates entropy; rough data give a negative total rate."""
    rng = np.random.default_rng(1)
    if dim == 1:
        w = wl.sine_1d(64)
        sch = _scheme(w)
        x = w["x"]
        rho = 0.5 + 0.3 * rng.uniform(size=64)
        U = thermo.prim_to_cons(sch.gas, rho, rng.uniform(-0.5, 0.5, (1, 64)), 1.0 + 0.2 * rng.uniform(size=64))
    else:
        w = wl.sine_2d(16)
        sch = _scheme(w)
        X, Y = w["x"]
        x = _wavy_mesh(X, Y)
        U = thermo.prim_to_cons(sch.gas, 0.5 + 0.3 * rng.uniform(size=X.shape),
                                rng.uniform(-0.5, 0.5, (2,) + X.shape), 1.0 + 0.2 * rng.uniform(size=X.shape))
    J = op.node_jacobian(sch, x)
    dU, dJ = op.rhs(sch, U * J, J, x, np.zeros_like(x))
    V = thermo.entropy_variables(sch.gas, U)
    terms = np.sum(V * dU, axis=0) - thermo.potential(sch.gas, U) * dJ
    assert terms.sum() < 0.0


def test_es_dissipation_sign_per_face():
    """At every face [[V]] . (F^ES - F^EC) <= 0 (the sign switch Y of Sec. 3.3)."""
    w = wl.sine_1d(48)
    sch = _scheme(w)
    sch_ec = _scheme(w, dissipation=False)
    rng = np.random.default_rng(2)
    rho = 0.4 + 0.6 * rng.uniform(size=48)
    U = thermo.prim_to_cons(sch.gas, rho, rng.uniform(-0.7, 0.7, (1, 48)), 0.8 + 0.6 * rng.uniform(size=48))
    Upad = op.pad(U, 3, 1, "periodic")
    Vpad = thermo.entropy_variables(sch.gas, Upad)
    n, xt = op.direction_metrics(sch, w["x"], np.zeros_like(w["x"]), 0, 3)
    F_es, _ = op.direction_fluxes(sch, Upad, n, xt, Vpad)
    F_ec, _ = op.direction_fluxes(sch_ec, Upad, n, xt, Vpad)
    jumpV = Vpad[:, 3:52] - Vpad[:, 2:51]            # faces i+1/2, i = -1..N-1
    prod = np.sum(jumpV * (F_es - F_ec), axis=0)
    assert np.all(prod <= 1e-12 * np.abs(jumpV).sum(axis=0) * np.abs(F_es).max())
    assert prod.min() < 0


def test_conservation_periodic():
    """The scheme is conservative: sum_i d(JU)_i/dt = 0 and sum_i dJ_i/dt = 0 on periodic data."""
    w = wl.sine_2d(16)
    sch = _scheme(w)
    X, Y = w["x"]
    x = _wavy_mesh(X, Y)
    J = op.node_jacobian(sch, x)
    U = _smooth_state(sch.gas, X, Y)
    xdot = 0.05 * np.stack([np.sin(2 * np.pi * (X + Y)), np.cos(2 * np.pi * (X - Y))])
    dU, dJ = op.rhs(sch, U * J, J, x, xdot)
    assert np.all(np.abs(dU.sum(axis=(1, 2))) < 1e-11 * np.abs(dU).sum(axis=(1, 2)).clip(min=1))
    assert abs(dJ.sum()) < 1e-12 * np.abs(dJ).sum()


# ------------------------------------------------------------- eigen-system

def _dUdV(g, U):
    """(dV/dU)^-1 with dV/dU from complex-step differentiation of V(U)."""
    n = U.shape[0]
    H = np.zeros((n, n))
    h = 1e-30
    for c in range(n):
        Uc = U.astype(complex)
        Uc[c] += 1j * h
        H[:, c] = np.imag(thermo.entropy_variables(g, Uc[:, None]))[:, 0] / h
    return np.linalg.inv(H)


@pytest.mark.parametrize("gname", ["units_a", "ideal"])
@pytest.mark.parametrize("dim", [1, 2])
def test_scaled_eigenvectors(gname, dim):
    """eq. eigen: R R^T = dU/dV and (dF_1/dU) R~ = R~ diag(lambda) (Sec. 3.3)."""
    g = thermo.gas_units_a() if gname == "units_a" else thermo.ideal_gas(1.4)
    rng = np.random.default_rng(3)
    for _ in range(10):
        rho = rng.uniform(0.3, 1.8)
        T = rng.uniform(1.05, 1.6)
        v = rng.uniform(-0.5, 0.5, dim)
        p = thermo.pressure(g, rho, T)
        U = thermo.prim_to_cons(g, np.array([rho]), v[:, None], np.array([p]))[:, 0]
        R, c = op.scaled_eigenvectors(g, np.array(rho), np.array(v[0]),
                                      None if dim == 1 else np.array(v[1]), np.array(p))
        R = R.reshape(dim + 2, dim + 2)
        assert np.allclose(R @ R.T, _dUdV(g, U), rtol=1e-8, atol=1e-8 * np.abs(R @ R.T).max())
        # flux Jacobian by complex step
        A = np.zeros((dim + 2, dim + 2))
        nvec = np.zeros((dim, 1))
        nvec[0] = 1.0
        for col in range(dim + 2):
            Uc = U.astype(complex)[:, None]
            Uc[col] += 1j * 1e-30
            A[:, col] = np.imag(thermo.flux(g, Uc, nvec))[:, 0] / 1e-30
        lam = [v[0] - c, v[0], v[0] + c] if dim == 1 else [v[0] - c, v[0], v[0], v[0] + c]
        assert np.allclose(A @ R, R @ np.diag(np.array(lam, dtype=float).ravel()), rtol=1e-9,
                           atol=1e-9 * np.abs(A @ R).max())


def test_rotation_invariance_of_dissipation_matrix():
    """T^T R(TU) R(TU)^T T = dU/dV(U): the rotated scaled eigenvectors give the same matrix."""
    g = thermo.gas_units_a()
    rho, T, v = 0.9, 1.3, np.array([0.3, -0.4])
    p = thermo.pressure(g, rho, T)
    U = thermo.prim_to_cons(g, np.array([rho]), v[:, None], np.array([p]))[:, 0]
    th = 0.7
    c, s = np.cos(th), np.sin(th)
    vn, vt = c * v[0] + s * v[1], -s * v[0] + c * v[1]
    R, _ = op.scaled_eigenvectors(g, np.array(rho), np.array(vn), np.array(vt), np.array(p))
    R = R.reshape(4, 4)
    Tm = np.array([[1, 0, 0, 0], [0, c, s, 0], [0, -s, c, 0], [0, 0, 0, 1.0]])
    assert np.allclose(Tm.T @ R @ R.T @ Tm, _dUdV(g, U), rtol=1e-8, atol=1e-8)


# --------------------------------------------------------------------- mesh

def test_filter_preserves_constants_and_sums():
    """Sec. 4 filter: the weights (1/2)^(|j|_1+d) sum to 1; on periodic data the total is kept."""
    rng = np.random.default_rng(4)
    om = rng.uniform(1, 3, (12, 15))
    out = mesh.low_pass(om, 2, ("periodic", "periodic"))
    assert np.isclose(out.sum(), om.sum(), rtol=1e-14)
    c = np.full((7, 9), 2.5)
    assert np.allclose(mesh.low_pass(c, 2, ("outflow", "outflow")), 2.5, rtol=1e-15)
    om1 = rng.uniform(1, 3, 20)
    assert np.isclose(mesh.low_pass(om1, 1, ("periodic",)).sum(), om1.sum(), rtol=1e-14)


def test_mm1_monitor_sees_the_density_only():
    """MM1 (Sec. 5: alpha_2 = alpha_3 = 0 in eq. van der Waalsmonitor): omega does not depend on G, and
    on a piecewise-linear density with slopes s_1 < s_2 it is sqrt(1 + alpha_1 (s / s_2)^2) away from
    the kink and the ends (second-order central differences are exact on linear data)."""
    x, d = wl.uniform_nodes(41, 0.0, 1.0, False)
    s1, s2 = 0.5, 2.0
    rho = np.where(x < 0.5, 1.0 + s1 * (x - 0.5), 1.0 + s2 * (x - 0.5))
    G = np.random.default_rng(7).uniform(-1.0, 1.0, x.shape)
    alphas = wl.mm1(wl.riemann_1d("RP1", n=41))["mesh"]["alphas"]
    assert alphas[1:] == (0.0, 0.0)
    om = mesh.monitor_vdw([rho, G], G, alphas, 1, ("outflow",), (d,))
    assert np.array_equal(om, mesh.monitor_vdw([rho, 0 * G], 0 * G, alphas, 1, ("outflow",), (d,)))
    left, right = slice(1, 19), slice(22, 40)
    assert np.allclose(om[left] ** 2 - 1.0, alphas[0] * (s1 / s2) ** 2, rtol=1e-12)
    assert np.allclose(om[right] ** 2 - 1.0, alphas[0], rtol=1e-12)


def _periodic_grid(dim, n=16):
    x1, d = wl.uniform_nodes(n, 0.0, 1.0, True)
    if dim == 1:
        return (x1,), (d,), ("periodic",)
    X, Y = np.meshgrid(x1, x1)
    return (X, Y), (d, d), ("periodic", "periodic")


@pytest.mark.parametrize("dim", [1, 2])
def test_vdw_monitor_closed_form(dim):
    """eq. van der Waalsmonitor with kappa = 2 (delta_1 = rho, delta_2 = G) on periodic sines.  Second-order central
    differences of sin(2 pi m xi) are cos(2 pi m xi) sin(2 pi m h)/h and -sin(2 pi m xi) 4 sin^2(pi m h)/h^2 exactly, so
    every normalised term is a trigonometric polynomial whose constant factor cancels against its maximum (n = 16
    puts nodes at the maxima).  With rho = 1 + 0.1 sin(4 pi xi_1) and G = 0.3 sum_k sin(2 pi xi_k):
    omega^2 = 1 + a1 cos^2(4 pi xi_1) + a2 mean_k cos^2(2 pi xi_k) + a3 mean_k sin^2(2 pi xi_k).
    The last term is |Delta_xi G|^2, the squared vector of second derivatives (Sec. 4); its gradient, or the term
    without the square, gives another function."""
    X, dxi, bc = _periodic_grid(dim)
    rho = 1.0 + 0.1 * np.sin(4 * np.pi * X[0])
    G = 0.3 * sum(np.sin(2 * np.pi * Xk) for Xk in X)
    a = (1200.0, 3000.0, 5000.0)
    om = mesh.monitor_vdw([rho, G], G, a, dim, bc, dxi)
    c2 = sum(np.cos(2 * np.pi * Xk) ** 2 for Xk in X) / dim
    s2 = sum(np.sin(2 * np.pi * Xk) ** 2 for Xk in X) / dim
    expect = 1.0 + a[0] * np.cos(4 * np.pi * X[0]) ** 2 + a[1] * c2 + a[2] * s2
    assert np.allclose(om**2, expect, rtol=1e-12, atol=0.0)
    # kappa = 1 (Example 5.4's MM): the second weight goes to |Delta_xi G|^2
    om1 = mesh.monitor_vdw([rho], G, (1200.0, 500.0), dim, bc, dxi)
    assert np.allclose(om1**2, 1.0 + 1200.0 * np.cos(4 * np.pi * X[0]) ** 2 + 500.0 * s2, rtol=1e-12, atol=0.0)


@pytest.mark.parametrize("dim", [1, 2])
def test_smooth_monitor_closed_form(dim):
    """eq. van der Waalssinmonitor (Example 5.1): omega^2 = 1 + a1 |grad rho|/max + a2 |Delta_xi rho|/max with the
    norms not squared.  For rho = 0.5 + 0.1 sum_k sin(2 pi xi_k) the exact difference quotients give
    |grad rho|/max = sqrt(mean_k cos^2(2 pi xi_k)) and |Delta_xi rho|/max = sqrt(mean_k sin^2(2 pi xi_k))."""
    X, dxi, bc = _periodic_grid(dim)
    rho = 0.5 + 0.1 * sum(np.sin(2 * np.pi * Xk) for Xk in X)
    om = mesh.monitor_smooth(rho, (20.0, 15.0), dim, bc, dxi)
    c = np.sqrt(sum(np.cos(2 * np.pi * Xk) ** 2 for Xk in X) / dim)
    s = np.sqrt(sum(np.sin(2 * np.pi * Xk) ** 2 for Xk in X) / dim)
    assert np.allclose(om**2, 1.0 + 20.0 * c + 15.0 * s, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2])
def test_sign_switch_dead_zone_leaves_real_jumps_alone(dim):
    """The dead zone of the sign switch Y (a plain jump within sign_tol of the size of the terms that form it has
    sign 0) only touches round-off-sized jumps: on rough random states, whose jumps are all far above 1e-12 of their
    scale, the operator with sign_tol = 1e-12 equals the paper's plain sign rule (sign_tol = 0) bit for bit."""
    if dim == 1:
        w = wl.sine_1d(48)
        shape = (48,)
    else:
        w = wl.sine_2d(20)
        shape = (20, 20)
    rho, v, p = wl.rough_state(shape, 17, dim)
    g = thermo.Gas(**w["gas"])
    out = []
    for tol in (1e-12, 0.0):
        sch = op.Scheme(gas=g, dim=dim, bc=w["bc"], dxi=w["dxi"], period=w["period"], sign_tol=tol)
        J = op.node_jacobian(sch, w["x"])
        JU = thermo.prim_to_cons(g, rho, v, p) * J
        out.append(op.rhs(sch, JU, J, w["x"], np.zeros_like(w["x"])))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_uniform_monitor_fixed_point():
    """With omega = const the uniform mesh solves the discrete mesh equation (x unchanged)."""
    w = wl.riemann_2d(12, moving=True)
    sch = _scheme(w)
    om = np.full(w["x"].shape[1:], 1.7)
    x, taken = mesh.jacobi(sch, w["x"], om, 4)
    assert np.allclose(x, w["x"], atol=1e-15) and taken == 4


def test_jacobi_1d_equidistribution():
    """A converged 1D mesh equidistributes omega: omega_{i+1/2} (x_{i+1} - x_i) is constant."""
    x0, d = wl.uniform_nodes(21, 0.0, 1.0, False)
    sch = op.Scheme(gas=thermo.gas_units_a(), dim=1, bc=("outflow",), dxi=(d,), period=(1.0,))
    om = 1.0 + 5.0 * np.exp(-50 * (x0 - 0.4) ** 2)
    x, _ = mesh.jacobi(sch, x0[None], om, 20000, eps=1e-15)
    flux = 0.5 * (om[1:] + om[:-1]) * np.diff(x[0])
    assert np.ptp(flux) < 1e-12 * flux.mean()


def test_limiter_keeps_order():
    """Delta_gamma limits every node to half of its spacing, so the mesh cannot fold."""
    x0, d = wl.uniform_nodes(30, 0.0, 1.0, False)
    sch = op.Scheme(gas=thermo.gas_units_a(), dim=1, bc=("outflow",), dxi=(d,), period=(1.0,))
    rng = np.random.default_rng(5)
    dx = rng.uniform(-3 * d, 3 * d, 30)
    dx[[0, -1]] = 0.0
    gam = mesh.limiter(sch, x0[None], dx[None])
    assert 0 < gam <= 1
    x1 = x0 + gam * dx
    assert np.all(np.diff(x1) > 0)
    # the bound is attained by some node
    moved = np.abs(gam * dx) / d
    assert moved.max() >= 0.5 - 1e-12 or gam == 1.0


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_cfl_on_a_translating_mesh(dim):
    """eq. cfl with the spectral radius of the xi_k flux Jacobian, |J xi_{k,t} + n_k . v| + L_k c over J: on a
    Cartesian mesh (n_k = e_k, J = 1) translating with constant velocity s (J xi_{k,t} = -s_k, eq. VCLCoeff), a
    uniform state gives Delta t = CFL / sum_k (|v_k - s_k| + c) / dxi_k; at rest s = 0."""
    n = (10, 12, 8)[:dim]
    dxi = tuple(1.0 / m for m in n)
    g = thermo.gas_units_a()
    sch = op.Scheme(gas=g, dim=dim, bc=("periodic",) * dim, dxi=dxi, period=(1.0,) * dim)
    axes = [np.arange(m) * h for m, h in zip(n, dxi)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]        # x_1 varies along the last axis
    x = np.stack(grids)
    shape = x.shape[1:]
    v = np.array([0.4, -0.3, 0.25])[:dim]
    s = np.array([0.9, 0.2, -0.6])[:dim]
    rho, p = 0.7, 1.1
    U = thermo.prim_to_cons(g, np.full(shape, rho), v.reshape((dim,) + (1,) * dim) * np.ones(shape), np.full(shape, p))
    J = np.ones(shape)
    c = np.sqrt(thermo.sound_speed2(g, rho, thermo.temperature(g, rho, p)))
    xdot = s.reshape((dim,) + (1,) * dim) * np.ones(shape)
    moving = 0.4 / sum((abs(v[k] - s[k]) + c) / dxi[k] for k in range(dim))
    rest = 0.4 / sum((abs(v[k]) + c) / dxi[k] for k in range(dim))
    assert stepper.cfl_dt(sch, U * J, J, x, 0.4, xdot) == pytest.approx(moving, rel=1e-13)
    assert stepper.cfl_dt(sch, U * J, J, x, 0.4) == pytest.approx(rest, rel=1e-13)


# ------------------------------------------------------------------ stepper

def test_ssp_rk3_order_conditions():
    """The Shu-Osher SSP-RK3 (Gottlieb, Shu & Tadmor) is third order: on du/dt = lambda u one
    step reproduces the Taylor polynomial 1 + z + z^2/2 + z^3/6, z = lambda dt."""
    A, B = stepper.RK3_A, stepper.RK3_B
    assert tuple(stepper.RK3_C) == (0.0, 1.0, 0.5)
    for lam, dt in ((-0.7, 0.1), (2.0, 0.05), (-3.0, 0.3)):
        u1 = A[0] + B[0] * (1 + dt * lam)
        u2 = A[1] * 1 + B[1] * (u1 + dt * lam * u1)
        u3 = A[2] * 1 + B[2] * (u2 + dt * lam * u2)
        z = lam * dt
        assert np.isclose(u3, 1 + z + z**2 / 2 + z**3 / 6, rtol=1e-15)
    # stage times: stage 2 sees U^n + dt L, stage 3 sees U^n + dt/4 (L1 + L2) -> t^n + dt/2


def test_design_order_1d_sine():
    """Example 5.1 setup on a fixed mesh with dt = CFL dxi^(5/3): the error in rho drops at ~5th order."""
    errs = []
    for n in (20, 40, 80):
        w = wl.sine_1d(n, t_end=0.05)
        sch = _scheme(w)
        J = op.node_jacobian(sch, w["x"])
        JU = thermo.prim_to_cons(sch.gas, w["rho"], w["v"], w["p"]) * J
        JU, J, x, _ = stepper.run(sch, stepper.MeshControl(), JU, J, w["x"], w["t_end"], 0.4,
                                  dt_fixed=0.4 * w["dxi"][0] ** (5 / 3))
        ex = 0.5 + 0.2 * np.sin(2 * np.pi * (x[0] - w["t_end"]))
        errs.append(np.abs(JU[0] / J - ex).mean())
    order = np.log2(errs[-2] / errs[-1])
    assert order > 4.5, errs


def test_design_order_1d_sine_moving_mesh():
    """Example 5.1's MM (smooth-test monitor, alpha = (20, 15), 20 filter passes, dt = CFL dxi^(5/3)):
    the error in rho at the moved nodes drops at ~5th order, as on the fixed mesh."""
    errs = []
    for n in (20, 40, 80):
        w = wl.sine_1d(n, t_end=0.05, moving=True)
        sch = _scheme(w)
        J = op.node_jacobian(sch, w["x"])
        JU = thermo.prim_to_cons(sch.gas, w["rho"], w["v"], w["p"]) * J
        mc = stepper.MeshControl(moving=True, **w["mesh"])
        JU, J, x, _ = stepper.run(sch, mc, JU, J, w["x"], w["t_end"], 0.4, dt_fixed=0.4 * w["dxi"][0] ** (5 / 3))
        assert np.abs(x - w["x"]).max() > 1e-3 * w["dxi"][0]          # the mesh did move
        ex = 0.5 + 0.2 * np.sin(2 * np.pi * (x[0] - w["t_end"]))
        errs.append(np.abs(JU[0] / J - ex).mean())
    order = np.log2(errs[-2] / errs[-1])
    assert order > 4.5, errs


def test_moving_mesh_step_runs_and_conserves():
    """One full MM step on the 1D sine (Example 5.1 monitor): mass is conserved on periodic data."""
    w = wl.sine_1d(40)
    sch = _scheme(w)
    J = op.node_jacobian(sch, w["x"])
    JU = thermo.prim_to_cons(sch.gas, w["rho"], w["v"], w["p"]) * J
    mc = stepper.MeshControl(moving=True, monitor="smooth", alphas=(20.0, 15.0), filter_passes=20,
                             sweeps=10)
    JU1, J1, x1, t1, info = stepper.step(sch, mc, JU, J, w["x"], 0.0, 1.0, 0.4)
    assert info["sweeps"] == 10 and 0 < info["gamma"] <= 1
    assert np.isclose(JU1.sum(axis=1), JU.sum(axis=1), rtol=1e-13).all()
    assert np.isclose(J1.sum(), J.sum(), rtol=1e-13)
    assert np.all(np.diff(x1[0]) > 0)
