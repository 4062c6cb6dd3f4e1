"""Pins of the oracle's 3D operator and mesh redistribution (Sec. 3 - Sec. 4 in three dimensions).

Each check ties the 3D code to something outside itself: exact metrics of polynomial maps,
reduction to the 2D and 1D operators (themselves pinned elsewhere), free-stream preservation
and entropy conservation, the eigen-system identities of eq. eigen, and separability of the
3D low-pass filter.
"""
import numpy as np
import pytest

from oracle import mesh, stepper, thermo
from oracle import operator as op
from paper_2407_05568_gb300 import workloads as wl


def _grid(n, lo=0.0, hi=1.0, periodic=True):
    x1, d = wl.uniform_nodes(n, lo, hi, periodic)
    Z, Y, X = np.meshgrid(x1, x1, x1, indexing="ij")
    return X, Y, Z, d


def _scheme3(d, bc="periodic", dissipation=True, gammas=(0.005, 0.045, 0.95)):
    return op.Scheme(gas=thermo.gas_units_a(), dim=3, bc=(bc,) * 3, dxi=(d, d, d), period=(1.0, 1.0, 1.0),
                     dissipation=dissipation, weno_gammas=gammas)


def _wavy3(X, Y, Z, amp=0.01):
    """Smooth periodic perturbation of the unit-cube mesh (x(X+1, .) = x + e_1 etc.)."""
    s = np.sin
    tp = 2 * np.pi
    return np.stack([X + amp * s(tp * X) * s(tp * Y) * np.cos(tp * Z),
                     Y + amp * s(tp * Y) * np.cos(tp * X) * s(tp * Z),
                     Z + amp * s(tp * Z) * s(tp * X + 0.3) * s(tp * Y)])


def _smooth_state3(g, X, Y, Z):
    tp = 2 * np.pi
    rho = 0.6 + 0.15 * np.sin(tp * X) * np.cos(tp * Y) + 0.05 * np.sin(tp * Z)
    v = np.stack([0.3 + 0.1 * np.cos(tp * Y), -0.2 + 0.1 * np.sin(tp * Z), 0.1 + 0.1 * np.sin(tp * X)])
    p = 1.0 + 0.1 * np.sin(tp * (Y + Z))
    return thermo.prim_to_cons(g, rho, v, p)


# ------------------------------------------------------------------ metrics

def test_metrics_exact_for_affine_and_quadratic_maps():
    """eq. SCLCoeff is exact for polynomial maps of low degree: for x = A xi + quadratic terms,
    J dxi_k/dx_j equals the cofactor (x_p)_{xi_l} (x_q)_{xi_m} - (x_p)_{xi_m} (x_q)_{xi_l} of
    the analytic Jacobian matrix at every node away from the ghost-dependent rim, and J its
    determinant (affine part)."""
    n = 16
    X, Y, Z, d = _grid(n, periodic=False)
    rng = np.random.default_rng(7)
    A = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    Q = 0.05 * rng.standard_normal((3, 3, 3))           # x_c += sum_ab Q[c,a,b] xi_a xi_b
    xi = np.stack([X, Y, Z])
    x = np.einsum("ca,a...->c...", A, xi) + np.einsum("cab,a...,b...->c...", Q, xi, xi)
    # analytic dx_c/dxi_a = A[c,a] + sum_b (Q[c,a,b] + Q[c,b,a]) xi_b
    M = A[:, :, None, None, None] + np.einsum("cab,b...->ca...", Q + Q.transpose(0, 2, 1), xi)
    sch = _scheme3(d, bc="outflow")
    inner = (slice(6, -6),) * 3
    for k in range(3):
        nk, _ = op.direction_metrics(sch, x, np.zeros_like(x), k, 0)
        l, m = (k + 1) % 3, (k + 2) % 3
        for j in range(3):
            p, q = (j + 1) % 3, (j + 2) % 3
            ref = M[p, l] * M[q, m] - M[p, m] * M[q, l]
            assert np.abs(nk[j][inner] - ref[inner]).max() < 1e-12, (k, j)
    # affine map: J = det A everywhere (ghosts by odd reflection are exact for linear maps)
    xa = np.einsum("ca,a...->c...", A, xi)
    J = op.node_jacobian(sch, xa)
    assert np.abs(J - np.linalg.det(A)).max() < 1e-12
    for k in range(3):
        nk, _ = op.direction_metrics(sch, xa, np.zeros_like(xa), k, 3)
        adj = np.linalg.det(A) * np.linalg.inv(A)          # adj[k, j] = J dxi_k/dx_j
        for j in range(3):
            assert np.abs(nk[j] - adj[k, j]).max() < 1e-12


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_discrete_scl_3d(bc):
    """eq. SCL_dis in 3D: with v = 0 and constant p the momentum right-hand side is -p times the
    SCL residual sum_k delta_k[J dxi_k/dx_j] of the face metric fluxes, which vanishes to round-off."""
    n = 12
    X, Y, Z, d = _grid(n, periodic=(bc == "periodic"))
    x = _wavy3(X, Y, Z, 0.02)
    sch = _scheme3(d, bc=bc, dissipation=False)
    g = sch.gas
    U = thermo.prim_to_cons(g, np.full_like(X, 0.8), np.zeros((3,) + X.shape), np.full_like(X, 1.0))
    J = op.node_jacobian(sch, x)
    dU, dJ = op.rhs(sch, U * J, J, x, np.zeros_like(x))
    assert np.abs(dU[1:4]).max() < 1e-12 / d
    assert np.abs(dJ).max() == 0.0


def test_free_stream_moving_mesh_3d():
    """A constant state stays constant on a moving 3D mesh: d(JU)/dt = U dJ/dt to round-off."""
    n = 12
    X, Y, Z, d = _grid(n)
    x = _wavy3(X, Y, Z)
    sch = _scheme3(d)
    g = sch.gas
    U0 = thermo.prim_to_cons(g, np.full_like(X, 0.8), np.stack([0.3 + 0 * X, -0.2 + 0 * X, 0.1 + 0 * X]),
                             np.full_like(X, 1.1))
    tp = 2 * np.pi
    xdot = 0.05 * np.stack([np.sin(tp * (X + Y)), np.cos(tp * (Y - Z)), np.sin(tp * (Z + X))])
    J = op.node_jacobian(sch, x)
    dU, dJ = op.rhs(sch, U0 * J, J, x, xdot)
    assert np.abs(dU - U0 * dJ).max() < 1e-12 * np.abs(U0).max() / d
    assert np.abs(dJ).max() > 1e-3


# ------------------------------------------------------------- reductions

def test_3d_reduces_to_2d():
    """State and mesh independent of xi_3, x_3 = xi_3, v_3 = 0: the 3D right-hand sides of
    (rho, m_1, m_2, E) and J equal the 2D operator's, and m_3's is zero (theta rotation only)."""
    n2, n3 = 16, 8
    x1, d = wl.uniform_nodes(n2, 0.0, 1.0, True)
    Y2, X2 = np.meshgrid(x1, x1, indexing="ij")
    tp = 2 * np.pi
    x2d = np.stack([X2 + 0.02 * np.sin(tp * X2) * np.sin(tp * Y2), Y2 + 0.02 * np.sin(tp * X2) * np.cos(tp * Y2)])
    xd2 = 0.05 * np.stack([np.sin(tp * (X2 + Y2)), np.cos(tp * (X2 - Y2))])
    g = thermo.gas_units_a()
    rng = np.random.default_rng(3)
    rho = 0.6 + 0.2 * np.sin(tp * X2) * np.cos(tp * Y2) + 0.02 * rng.standard_normal(X2.shape)
    v2 = np.stack([0.3 + 0.1 * np.cos(tp * Y2), -0.2 + 0.1 * np.sin(tp * X2)])
    p = 1.0 + 0.1 * np.sin(tp * Y2)
    U2 = thermo.prim_to_cons(g, rho, v2, p)
    s2 = op.Scheme(gas=g, dim=2, bc=("periodic",) * 2, dxi=(d, d), period=(1.0, 1.0))
    J2 = op.node_jacobian(s2, x2d)
    dU2, dJ2 = op.rhs(s2, U2 * J2, J2, x2d, xd2)

    z1, dz = wl.uniform_nodes(n3, 0.0, 1.0, True)
    rep = lambda a: np.broadcast_to(a, (n3,) + a.shape).copy()
    Z = np.broadcast_to(z1[:, None, None], (n3, n2, n2)).copy()
    x3 = np.stack([rep(x2d[0]), rep(x2d[1]), Z])
    xd3 = np.stack([rep(xd2[0]), rep(xd2[1]), np.zeros_like(Z)])
    v3 = np.stack([rep(v2[0]), rep(v2[1]), np.zeros_like(Z)])
    U3 = thermo.prim_to_cons(g, rep(rho), v3, rep(p))
    s3 = op.Scheme(gas=g, dim=3, bc=("periodic",) * 3, dxi=(d, d, dz), period=(1.0, 1.0, 1.0))
    J3 = op.node_jacobian(s3, x3)
    assert np.abs(J3 - rep(J2)).max() < 1e-13
    dU3, dJ3 = op.rhs(s3, U3 * J3, J3, x3, xd3)
    scale = np.abs(dU2).max()
    for c3, c2 in ((0, 0), (1, 1), (2, 2), (4, 3)):
        assert np.abs(dU3[c3] - rep(dU2[c2])).max() < 1e-11 * scale, c3
    assert np.abs(dU3[3]).max() < 1e-11 * scale
    assert np.abs(dJ3 - rep(dJ2)).max() < 1e-11 * np.abs(dJ2).max()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_3d_reduces_to_1d_along_each_axis(axis):
    """A rough state varying along x_axis only with velocity along it, Cartesian mesh: the 3D
    right-hand side on every line equals the 1D operator's (for x_3 this is the frame theta = 0,
    phi = pi/2 of a face normal along x_3)."""
    n, m = 24, 6
    g = thermo.gas_units_a()
    x1, d = wl.uniform_nodes(n, 0.0, 1.0, True)
    rng = np.random.default_rng(11 + axis)
    rho = 0.7 + 0.3 * rng.uniform(size=n)
    u = 0.3 * rng.standard_normal(n)
    p = 1.0 + 0.3 * rng.uniform(size=n)
    s1 = op.Scheme(gas=g, dim=1, bc=("periodic",), dxi=(d,), period=(1.0,))
    U1 = thermo.prim_to_cons(g, rho, u[None], p)
    J1 = op.node_jacobian(s1, x1[None])
    dU1, _ = op.rhs(s1, U1 * J1, J1, x1[None], np.zeros((1, n)))

    shape = [m, m, m]
    shape[2 - axis] = n
    o1, do = wl.uniform_nodes(m, 0.0, 1.0, True)
    coords = []
    for k in range(3):
        line = x1 if k == axis else o1
        sh = [1, 1, 1]
        sh[2 - k] = line.size
        coords.append(np.broadcast_to(line.reshape(sh), shape).copy())
    x3 = np.stack(coords)
    along = lambda a: np.broadcast_to(a.reshape([n if 2 - k == 2 - axis else 1 for k in range(2, -1, -1)]),
                                      shape).copy()
    v3 = np.zeros((3,) + tuple(shape))
    v3[axis] = along(u)
    dxi = [do, do, do]
    dxi[axis] = d
    s3 = op.Scheme(gas=g, dim=3, bc=("periodic",) * 3, dxi=tuple(dxi), period=(1.0, 1.0, 1.0))
    U3 = thermo.prim_to_cons(g, along(rho), v3, along(p))
    J3 = op.node_jacobian(s3, x3)
    dU3, dJ3 = op.rhs(s3, U3 * J3, J3, x3, np.zeros_like(x3))
    scale = np.abs(dU1).max()
    for c3, c1 in ((0, 0), (1 + axis, 1), (4, 2)):
        assert np.abs(dU3[c3] - along(dU1[c1])).max() < 1e-11 * scale, c3
    for t in range(3):
        if t != axis:
            assert np.abs(dU3[1 + t]).max() < 1e-11 * scale
    assert np.abs(dJ3).max() == 0.0


# ------------------------------------------------------------------ entropy

def test_ec_scheme_conserves_entropy_3d():
    """Without dissipation the 3D scheme conserves the total entropy on a moving periodic mesh
    (Sec. 3.2): the rate is round-off against the size of its terms."""
    n = 12
    X, Y, Z, d = _grid(n)
    x = _wavy3(X, Y, Z)
    sch = _scheme3(d, dissipation=False)
    U = _smooth_state3(sch.gas, X, Y, Z)
    J = op.node_jacobian(sch, x)
    tp = 2 * np.pi
    xdot = 0.05 * np.stack([np.sin(tp * (X + Y)), np.cos(tp * (Y - Z)), np.sin(tp * (Z + X))])
    dU, dJ = op.rhs(sch, U * J, J, x, xdot)
    rate = op.entropy_rate(sch, U * J, J, dU, dJ)
    V = thermo.entropy_variables(sch.gas, U)
    size = d**3 * float(np.sum(np.abs(V * dU)))
    assert abs(rate) < 1e-12 * size


def test_es_scheme_produces_entropy_3d():
    """With the dissipation of eq. HOstable the total entropy of a rough state decreases."""
    n = 10
    X, Y, Z, d = _grid(n)
    sch = _scheme3(d)
    g = sch.gas
    rng = np.random.default_rng(5)
    rho = 0.7 + 0.4 * rng.uniform(size=X.shape)
    v = 0.3 * rng.standard_normal((3,) + X.shape)
    p = 1.0 + 0.4 * rng.uniform(size=X.shape)
    U = thermo.prim_to_cons(g, rho, v, p)
    x = _wavy3(X, Y, Z)
    J = op.node_jacobian(sch, x)
    dU, dJ = op.rhs(sch, U * J, J, x, np.zeros_like(x))
    assert op.entropy_rate(sch, U * J, J, dU, dJ) < 0.0


# ------------------------------------------------------------ eigen-system

def _dUdV(g, U):
    h = 1e-30
    H = np.zeros((U.size, U.size))
    for c in range(U.size):
        Uc = U.astype(complex)
        Uc[c] += 1j * h
        H[:, c] = np.imag(thermo.entropy_variables(g, Uc[:, None]))[:, 0] / h
    return np.linalg.inv(H)


@pytest.mark.parametrize("gname", ["units_a", "ideal"])
def test_scaled_eigenvectors_3d(gname):
    """eq. eigen in 3D: R R^T = dU/dV and (dF_1/dU) R~ = R~ diag(v - c, v, v, v, v + c)."""
    g = thermo.gas_units_a() if gname == "units_a" else thermo.ideal_gas(1.4)
    rng = np.random.default_rng(9)
    for _ in range(8):
        rho = rng.uniform(0.3, 1.8)
        T = rng.uniform(1.05, 1.6)
        v = rng.uniform(-0.5, 0.5, 3)
        p = thermo.pressure(g, rho, T)
        U = thermo.prim_to_cons(g, np.array([rho]), v[:, None], np.array([p]))[:, 0]
        R, c = op.scaled_eigenvectors(g, np.array(rho), np.array(v[0]), (np.array(v[1]), np.array(v[2])),
                                      np.array(p))
        R = R.reshape(5, 5)
        assert np.allclose(R @ R.T, _dUdV(g, U), rtol=1e-8, atol=1e-8 * np.abs(R @ R.T).max())
        A = np.zeros((5, 5))
        nvec = np.array([[1.0], [0.0], [0.0]])
        for col in range(5):
            Uc = U.astype(complex)[:, None]
            Uc[col] += 1j * 1e-30
            A[:, col] = np.imag(thermo.flux(g, Uc, nvec))[:, 0] / 1e-30
        lam = np.array([v[0] - c, v[0], v[0], v[0], v[0] + c], dtype=float).ravel()
        assert np.allclose(A @ R, R @ np.diag(lam), rtol=1e-9, atol=1e-9 * np.abs(A @ R).max())


def test_frame_3d_rotation():
    """T of Sec. 3.3 in 3D is orthogonal with first row n/L; the rotated scaled eigenvectors
    give T^T R R^T T = dU/dV for arbitrary normals, including n along x_3 (theta = 0)."""
    g = thermo.gas_units_a()
    rng = np.random.default_rng(2)
    rho, T = 0.9, 1.3
    v = np.array([0.3, -0.4, 0.2])
    p = thermo.pressure(g, rho, T)
    U = thermo.prim_to_cons(g, np.array([rho]), v[:, None], np.array([p]))[:, 0]
    normals = [rng.standard_normal(3) for _ in range(5)] + [np.array([0.0, 0.0, 2.0]), np.array([0.0, 0.0, -1.5])]
    for nv in normals:
        L, fr = op.frame_3d(nv[:, None])
        F = fr[:, :, 0]
        assert np.allclose(F @ F.T, np.eye(3), atol=1e-15)
        assert np.allclose(F[0], nv / np.linalg.norm(nv), atol=1e-15)
        assert np.isclose(L[0], np.linalg.norm(nv))
        vr = F @ v
        R, _ = op.scaled_eigenvectors(g, np.array(rho), np.array(vr[0]), (np.array(vr[1]), np.array(vr[2])),
                                      np.array(p))
        R = R.reshape(5, 5)
        Tm = np.eye(5)
        Tm[1:4, 1:4] = F
        assert np.allclose(Tm.T @ R @ R.T @ Tm, _dUdV(g, U), rtol=1e-8, atol=1e-8)


# --------------------------------------------------------------------- mesh

def test_filter_3d_is_separable():
    """The 3D filter weights (1/2)^(|j|_1 + 3) factor into (1/4, 1/2, 1/4) per direction: one 3D
    pass equals three 1D passes, and the weights sum to 1."""
    rng = np.random.default_rng(4)
    om = rng.uniform(1, 3, (6, 7, 8))
    bc = ("periodic",) * 3
    out = mesh.low_pass(om, 3, bc)
    sep = om
    for ax in range(3):
        sep = 0.25 * np.roll(sep, 1, axis=ax) + 0.5 * sep + 0.25 * np.roll(sep, -1, axis=ax)
    assert np.allclose(out, sep, rtol=1e-15, atol=0)
    assert np.allclose(mesh.low_pass(np.full((5, 6, 7), 2.5), 3, ("outflow",) * 3), 2.5, rtol=1e-15)


def test_uniform_monitor_fixed_point_3d():
    """With omega = const the uniform 3D mesh solves the discrete mesh equation."""
    X, Y, Z, d = _grid(8, periodic=False)
    sch = _scheme3(d, bc="outflow")
    x = np.stack([X, Y, Z])
    xn, taken = mesh.jacobi(sch, x, np.full(X.shape, 1.7), 3)
    assert np.allclose(xn, x, atol=1e-15) and taken == 3


def test_jacobi_3d_converges_to_1d_equidistribution():
    """omega varying along xi_1 only (outflow along xi_1, periodic across): the converged 3D
    mesh equidistributes omega along every xi_1 line, omega_{i+1/2} (x_{i+1} - x_i) = const, and
    x_2, x_3 stay put."""
    n, m = 16, 4
    x1, d = wl.uniform_nodes(n, 0.0, 1.0, False)
    o1, do = wl.uniform_nodes(m, 0.0, 1.0, True)
    Z, Y, X = np.meshgrid(o1, o1, x1, indexing="ij")
    om1 = 1.0 + 4.0 * np.exp(-40 * (x1 - 0.35) ** 2)
    s3 = op.Scheme(gas=thermo.gas_units_a(), dim=3, bc=("outflow", "periodic", "periodic"), dxi=(d, do, do),
                   period=(1.0,) * 3)
    x3n, taken = mesh.jacobi(s3, np.stack([X, Y, Z]), np.broadcast_to(om1, X.shape).copy(), 100000, eps=1e-15)
    assert taken < 100000
    flux = 0.5 * (om1[1:] + om1[:-1]) * np.diff(x3n[0], axis=-1)
    assert np.ptp(flux) < 1e-12 * flux.mean()
    assert np.abs(x3n[1] - Y).max() < 1e-15 and np.abs(x3n[2] - Z).max() < 1e-15


def test_moving_mesh_step_3d_keeps_free_stream_and_conserves():
    """One full 3D moving-mesh step (CFL, monitor, filter, Jacobi, limiter, three RK stages) on a
    periodic sine wave: the total of each conserved variable is kept and the mesh moved (two
    filter passes: twenty flatten the monitor of a 10-node wave to round-off)."""
    w = wl.sine_3d(10, moving=True)
    w["mesh"] = dict(w["mesh"], filter_passes=2)
    g = thermo.Gas(**w["gas"])
    sch = op.Scheme(gas=g, dim=3, bc=w["bc"], dxi=w["dxi"], period=w["period"], weno_gammas=w["weno_gammas"])
    J = op.node_jacobian(sch, w["x"])
    JU = thermo.prim_to_cons(g, w["rho"], w["v"], w["p"]) * J
    mc = stepper.MeshControl(moving=True, **w["mesh"])
    JU1, J1, x1, t1, info = stepper.step(sch, mc, JU, J, w["x"], 0.0, 1.0, 0.4)
    assert info["sweeps"] == 10 and 0.0 < info["gamma"] <= 1.0
    assert np.abs(x1 - w["x"]).max() > 1e-6
    assert np.allclose(JU1.sum(axis=(1, 2, 3)), JU.sum(axis=(1, 2, 3)), rtol=1e-13, atol=1e-13)
    assert np.isclose(J1.sum(), J.sum(), rtol=1e-13)


def test_sign_switch_ignores_velocity_noise_where_v_t_is_zero():
    """Where the exact tangential velocity is zero, velocity noise at the level of rounding (1e-18)
    must not turn on the tangential waves' dissipation: the dead zone of Y counts the tangential
    entry of R as |v_t| + c (round-off in a velocity follows the flow's velocity scale)."""
    n = 14
    X, Y, Z, d = _grid(n, periodic=False)
    sch = _scheme3(d, bc="outflow")
    g = sch.gas
    inside = X**2 + Y**2 + Z**2 < 0.25
    U0 = thermo.prim_to_cons(g, np.where(inside, 1.2, 0.6), np.zeros((3,) + X.shape), np.where(inside, 1.8, 1.0))
    x = np.stack([X, Y, Z])
    J = op.node_jacobian(sch, x)
    # one stage: the flow starts at the sphere, the far field keeps v = 0 exactly
    dt = 0.5 * stepper.cfl_dt(sch, U0 * J, J, x, 0.4)
    JU1, J1 = stepper.rk_stage(sch, 0, dt, U0 * J, J, U0 * J, J, x, np.zeros_like(x))
    still = np.all(JU1[1:4] == 0.0, axis=0)
    assert still.any() and not still.all()
    rng = np.random.default_rng(1)
    JUn = JU1.copy()
    JUn[1:4] += np.where(still, 1e-18 * rng.standard_normal((3,) + X.shape), 0.0)
    dU, _ = op.rhs(sch, JU1, J1, x, np.zeros_like(x))
    dUn, _ = op.rhs(sch, JUn, J1, x, np.zeros_like(x))
    assert np.abs(dUn - dU).max() < 1e-12 * np.abs(dU).max()


def test_frame_angle_ignores_rounding_of_vanishing_metrics():
    """The 3D face frame takes theta = 0 when |(n_1, n_2)| <= 1e-12 |n|.  On an outflow box whose boundary planes
    stay Cartesian (the mesh velocity vanishes on the boundary nodes, as the mesh solve makes it) the
    x_3-faces' (n_1, n_2) are the rounding of exact zeros; with theta taken from that rounding the
    tangential frame, and through the per-field sign switch the dissipation, followed the noise (1e-5
    relative changes of the right-hand side under 1-ulp changes of the mesh).  Now the operator is as
    insensitive to such changes as on any other mesh."""
    from oracle import operator as op
    L, fr = op.frame_3d(np.array([[3e-15, 0.0], [-2e-15, 1e-10], [1.0, 1.0]]))
    assert np.array_equal(fr[1][:, 0], [0.0, 1.0, 0.0])            # e_t1 with theta = 0
    assert abs(fr[1][0, 1] + 1.0) < 1e-12                             # a 1e-10 tilt keeps its angle (pi/2)
    X = [wl.uniform_nodes(10, 0.0, 1.0, False)[0]] * 3
    Z, Y, Xg = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    rng = np.random.default_rng(21)
    rho = 0.6 + 0.1 * rng.random(Xg.shape)
    p = 1.0 + 0.1 * rng.random(Xg.shape)
    v = 0.1 * rng.standard_normal((3,) + Xg.shape)
    g = thermo.gas_units_a()
    d = 1.0 / 9.0
    sch = op.Scheme(gas=g, dim=3, bc=("outflow",) * 3, dxi=(d, d, d), period=(1.0, 1.0, 1.0))
    x = np.stack([Xg, Y, Z])
    tp = 2 * np.pi
    xd = 0.05 * np.stack([np.sin(tp * (Xg + Y)), np.cos(tp * (Y - Z)), np.sin(tp * (Z + Xg))])
    for ax in (1, 2, 3):
        for e in (0, -1):
            idx = [slice(None)] * 4
            idx[ax] = e
            xd[tuple(idx)] = 0.0
    xs = x + 1e-3 * xd
    J = op.node_jacobian(sch, xs)
    JU = thermo.prim_to_cons(g, rho, v, p) * J
    d0, _ = op.rhs(sch, JU, J, xs, xd)
    d1, _ = op.rhs(sch, JU, J, xs * (1.0 + 2e-16 * rng.standard_normal(xs.shape)), xd)
    assert np.abs(d1 - d0).sum() < 1e-12 * np.abs(d0).sum()


def test_example_5_7_runs_to_its_final_time():
    """Example 5.7 (Table 5.1's RP1 states inside and outside a sphere of radius 0.5; MM with Example 5.5's
    monitor) at 12^3 on the moving mesh, with the paper's 3D CFL of 0.3: every node stays admissible after every
    step up to the example's final time (t = 0.2 in the paper's reduced units), and, as in RP1, G < 0 appears
    between the rarefaction and the shock.  Taking eq. cfl's spectral radius with the mesh at rest instead of with
    the step's mesh velocity, the first step already left the admissible region."""
    w = wl.spherical_shock_3d(12)
    assert w["cfl"] == 0.3 and w["t_end"] == pytest.approx(0.2 * np.sqrt(3.0 / 8.0))
    g = thermo.Gas(**w["gas"])
    sch = op.Scheme(gas=g, dim=3, bc=tuple(w["bc"]), dxi=tuple(w["dxi"]), period=tuple(w["period"]))
    mc = stepper.MeshControl(moving=True, **w["mesh"])
    x = w["x"]
    J = op.node_jacobian(sch, x)
    JU = thermo.prim_to_cons(g, w["rho"], w["v"], w["p"]) * J
    t, steps = 0.0, 0
    while t < w["t_end"] * (1.0 - 1e-14):
        JU, J, x, t, info = stepper.step(sch, mc, JU, J, x, t, w["t_end"], w["cfl"])
        steps += 1
        rho, v, T, p = thermo.cons_to_prim(g, JU / J)
        assert thermo.admissible(g, rho, T).all(), steps
    assert steps > 30
    assert np.abs(x - w["x"]).max() > 0.1 * w["dxi"][0]                  # the mesh moved
    assert thermo.fundamental_derivative(g, rho, T).min() < -0.1
