"""Adaptive mesh redistribution (oracle; test infrastructure only).

Sec. 4: the mesh follows the Winslow equation div_xi(omega grad_xi x_k) = 0
(eq. mesh_EL), solved by Jacobi sweeps of its second-order central
discretisation, with the monitor omega of eq. van der Waalsmonitor (or the
smooth-test monitor eq. van der Waalssinmonitor of Example 5.1), smoothed by
the low-pass filter of Sec. 4, and the node movement limited by Delta_gamma.

Readings of points the paper leaves open:
  * gradients and second derivatives of the monitor use second-order central
    differences on the computational mesh (the order of Sec. 4's mesh
    equation); a term whose normalising maximum is 0 is dropped;
  * monitor and filter ghosts: periodic = wrap, outflow = copy, wall / symmetry = mirror;
  * at most mu sweeps are taken; with eps > 0 the sweeps stop as soon as
    max |x^[nu+1] - x^[nu]| < eps;
  * nodes on an outflow boundary stay fixed; nodes on a wall or symmetry plane slide along it
    (their normal coordinate stays); periodic boundary nodes move;
  * Delta_gamma = min(1, the bounds of Sec. 4 over all nodes and directions).
"""
import numpy as np

from .operator import PERIODIC, axis_of, mirrored, pad, pad_coords


def _shift(a, k, dim, bc, s):
    """a at node i + s e_k (s = +1 / -1) with ghosts by the boundary condition."""
    ax = axis_of(k, dim)
    ap = pad(a, 1, ax, bc[k])
    n = a.shape[ax]
    return np.take(ap, np.arange(1 + s, 1 + s + n), axis=ax)


def grad_sq(a, dim, bc, dxi):
    """|grad_xi a|^2 with second-order central differences."""
    out = np.zeros_like(a)
    for k in range(dim):
        d = (_shift(a, k, dim, bc, 1) - _shift(a, k, dim, bc, -1)) / (2.0 * dxi[k])
        out += d * d
    return out


def second_sq(a, dim, bc, dxi):
    """|Delta_xi a|^2 where Delta_xi a = (d^2 a/d xi_1^2, ..., d^2 a/d xi_d^2) (Sec. 4)."""
    out = np.zeros_like(a)
    for k in range(dim):
        d = (_shift(a, k, dim, bc, 1) - 2.0 * a + _shift(a, k, dim, bc, -1)) / dxi[k] ** 2
        out += d * d
    return out


def _normalised(t):
    m = np.max(t)
    return t / m if m > 0.0 else np.zeros_like(t)


def monitor_vdw(fields, G, alphas, dim, bc, dxi):
    """eq. van der Waalsmonitor: omega = (1 + sum_k alpha_k |grad delta_k|^2/max + alpha_{k+1} |Delta G|^2/max)^(1/2).

    fields = [delta_1, ..., delta_kappa]; alphas has kappa + 1 entries.
    """
    s = np.ones_like(G)
    for a_k, f in zip(alphas[:len(fields)], fields):
        s = s + a_k * _normalised(grad_sq(f, dim, bc, dxi))
    s = s + alphas[len(fields)] * _normalised(second_sq(G, dim, bc, dxi))
    return np.sqrt(s)


def monitor_smooth(rho, alphas, dim, bc, dxi):
    """eq. van der Waalssinmonitor: omega = (1 + a1 |grad rho|/max + a2 |Delta rho|/max)^(1/2)."""
    t1 = _normalised(np.sqrt(grad_sq(rho, dim, bc, dxi)))
    t2 = _normalised(np.sqrt(second_sq(rho, dim, bc, dxi)))
    return np.sqrt(1.0 + alphas[0] * t1 + alphas[1] * t2)


def low_pass(omega, dim, bc):
    """One pass of omega_i <- sum_{j in {0,+-1}^d} (1/2)^(|j|_1 + d) omega_{i+j} (Sec. 4)."""
    out = np.zeros_like(omega)
    if dim == 1:
        for s in (-1, 0, 1):
            nb = omega if s == 0 else _shift(omega, 0, 1, bc, s)
            out += 0.5 ** (abs(s) + 1) * nb
        return out
    if dim == 3:
        for s3 in (-1, 0, 1):
            pl = omega if s3 == 0 else _shift(omega, 2, 3, bc, s3)
            for s2 in (-1, 0, 1):
                row = pl if s2 == 0 else _shift(pl, 1, 3, bc, s2)
                for s1 in (-1, 0, 1):
                    nb = row if s1 == 0 else _shift(row, 0, 3, bc, s1)
                    out += 0.5 ** (abs(s1) + abs(s2) + abs(s3) + 3) * nb
        return out
    for s2 in (-1, 0, 1):
        row = omega if s2 == 0 else _shift(omega, 1, 2, bc, s2)
        for s1 in (-1, 0, 1):
            nb = row if s1 == 0 else _shift(row, 0, 2, bc, s1)
            out += 0.5 ** (abs(s1) + abs(s2) + 2) * nb
    return out


def _fixed_mask(shape, dim, bc):
    """Per coordinate component, True where it does not move: every component on an outflow
    boundary, the normal component on a wall or symmetry plane (its nodes slide along it)."""
    fixed = np.zeros((dim,) + tuple(shape), dtype=bool)
    for k in range(dim):
        if bc[k] == PERIODIC:
            continue
        ax = axis_of(k, dim)
        for end, mir in zip((0, -1), mirrored(bc[k])):
            idx = [slice(None)] * dim
            idx[ax] = end
            comps = [k] if mir else list(range(dim))
            for c in comps:
                fixed[c][tuple(idx)] = True
    return fixed


def jacobi(sch, x0, omega, mu, eps=0.0):
    """Jacobi iteration for the discrete mesh equation (Sec. 4).

    x^[nu+1]_i = sum_k (omega_{k,+1/2} x^[nu]_{i+e_k} + omega_{k,-1/2} x^[nu]_{i-e_k}) / dxi_k^2
                 / sum_k (omega_{k,+1/2} + omega_{k,-1/2}) / dxi_k^2,
    omega_{k,+-1/2} = (omega_i + omega_{i+-e_k})/2.  Returns (x^[nu_end], sweeps taken).
    """
    dim = sch.dim
    bc = sch.bc
    fixed = _fixed_mask(x0.shape[1:], dim, bc)
    wp = [0.5 * (omega + _shift(omega, k, dim, bc, 1)) for k in range(dim)]
    wm = [0.5 * (omega + _shift(omega, k, dim, bc, -1)) for k in range(dim)]
    den = sum((wp[k] + wm[k]) / sch.dxi[k] ** 2 for k in range(dim))
    x = x0.copy()
    taken = 0
    for _ in range(mu):
        xp = pad_coords(sch, x, 1)
        new = np.empty_like(x)
        for c in range(dim):
            num = np.zeros_like(den)
            for k in range(dim):
                ax = axis_of(k, dim)
                n = x.shape[1 + ax]
                sl_other = [slice(1, -1)] * dim
                hi = list(sl_other)
                lo = list(sl_other)
                hi[ax] = slice(2, 2 + n)
                lo[ax] = slice(0, n)
                num += (wp[k] * xp[c][tuple(hi)] + wm[k] * xp[c][tuple(lo)]) / sch.dxi[k] ** 2
            new[c] = np.where(fixed[c], x[c], num / den)
        change = float(np.max(np.abs(new - x)))
        x = new
        taken += 1
        if eps > 0.0 and change < eps:
            break
    return x, taken


def limiter(sch, xn, dx):
    """Delta_gamma of Sec. 4: each node may move at most half of its spacing to the neighbour it moves towards.

    Delta_gamma <= -(x_k^n(i) - x_k^n(i - e_k)) / (2 dx_k(i))  where dx_k(i) < 0,
    Delta_gamma <=  (x_k^n(i + e_k) - x_k^n(i)) / (2 dx_k(i))  where dx_k(i) > 0;
    the result is the minimum over all nodes and directions, and at most 1.
    """
    dim = sch.dim
    xp = pad_coords(sch, xn, 1)
    gam = 1.0
    for k in range(dim):
        ax = axis_of(k, dim)
        n = xn.shape[1 + ax]
        sl = [slice(1, -1)] * dim
        hi = list(sl)
        lo = list(sl)
        hi[ax] = slice(2, 2 + n)
        lo[ax] = slice(0, n)
        xk = xn[k]
        d = dx[k]
        neg = d < 0.0
        pos = d > 0.0
        safe = np.where(d == 0.0, 1.0, d)
        if np.any(neg):
            b = -(xk - xp[k][tuple(lo)]) / (2.0 * safe)
            gam = min(gam, float(np.min(b[neg])))
        if np.any(pos):
            b = (xp[k][tuple(hi)] - xk) / (2.0 * safe)
            gam = min(gam, float(np.min(b[pos])))
    return gam
