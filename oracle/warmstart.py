"""Mesh solve with a warm start (oracle; test infrastructure only).

The Jacobi iteration of Sec. 4 solves the discretised mesh equation with the
monitor omega frozen at the current mesh x^n.  A warm start x_s changes only
where the iteration starts; this module states how a start is assessed and
continued, and what features a network sees:

  * features: ln(omega) (omega after the filter passes), G/(1 + |G|) with the
    fundamental derivative G of Sec. 1, and the displacement of x^n from the
    Cartesian mesh (x_00 + i dxi_1, y_00 + j dxi_2) in cells;
  * warm start from a network output o (cells): x_s = x^n + dxi_k o_k at nodes
    that move, x^n at fixed (boundary) coordinates and where o is not finite;
  * guarded solve: the first sweep runs from x^n and from x_s, changing the mesh
    by c0 and c1 (max norm); x_s is continued if c1 < kappa c0 (kappa = the
    guard ratio), else x^n; the sweeps then stop as in ``mesh.jacobi`` (eps, at
    most mu sweeps in total on the continued path, the guarded first sweep
    counting once).  kappa > 1 admits a start whose first residual is larger
    but which is closer to where the iteration ends; a start with noise at the
    grid scale (which the plain Jacobi sweep does not damp: the checkerboard
    mode only flips sign) has c1 many times c0 and is refused.

The guard and the features are this implementation's design, not the paper's.
"""
import numpy as np

from . import mesh, thermo


def filtered_monitor(sch, mc, JU, J):
    """omega of Sec. 4 after mc.filter_passes passes of the low-pass filter, and G."""
    g = sch.gas
    rho, v, T, p = thermo.cons_to_prim(g, JU / J)
    G = thermo.fundamental_derivative(g, rho, T)
    if mc.monitor == "smooth":
        om = mesh.monitor_smooth(rho, mc.alphas, sch.dim, sch.bc, sch.dxi)
    else:
        om = mesh.monitor_vdw([rho, G][:mc.kappa], G, mc.alphas, sch.dim, sch.bc, sch.dxi)
    for _ in range(mc.filter_passes):
        om = mesh.low_pass(om, sch.dim, sch.bc)
    return om, G


def features(sch, mc, JU, J, x):
    """[ln omega, G/(1+|G|), (x - x_00 - i dxi_1)/dxi_1, (y - y_00 - j dxi_2)/dxi_2] (2D)."""
    om, G = filtered_monitor(sch, mc, JU, J)
    n2, n1 = x.shape[1:]
    i = np.arange(n1)[None, :]
    j = np.arange(n2)[:, None]
    d1 = (x[0] - (x[0, 0, 0] + i * sch.dxi[0])) / sch.dxi[0]
    d2 = (x[1] - (x[1, 0, 0] + j * sch.dxi[1])) / sch.dxi[1]
    return np.stack([np.log(om), G / (1.0 + np.abs(G)), d1, d2])


def warm_start(sch, xn, out):
    """x_s = x^n + dxi_k out_k at moving nodes; fixed coordinates and non-finite outputs keep x^n."""
    fixed = mesh._fixed_mask(xn.shape[1:], sch.dim, sch.bc)
    xs = xn.copy()
    for k in range(sch.dim):
        ok = ~fixed[k] & np.isfinite(out[k])
        xs[k] = np.where(ok, xn[k] + sch.dxi[k] * np.where(ok, out[k], 0.0), xn[k])
    return xs


def solve(sch, mc, JU, J, xn, x_start=None, guard_ratio=1.0):
    """The mesh solve of Sec. 4 without the limiter: (x^[nu], sweeps, picked)."""
    om, _ = filtered_monitor(sch, mc, JU, J)
    if x_start is None or mc.sweeps == 0:
        x, k = mesh.jacobi(sch, xn, om, mc.sweeps, mc.eps)
        return x, k, 0
    x0, _ = mesh.jacobi(sch, xn, om, 1)
    x1, _ = mesh.jacobi(sch, x_start, om, 1)
    c0 = float(np.max(np.abs(x0 - xn)))
    c1 = float(np.max(np.abs(x1 - x_start)))
    picked = 1 if c1 < guard_ratio * c0 else 0
    x = x1 if picked else x0
    c = c1 if picked else c0
    if mc.eps > 0.0 and c < mc.eps:
        return x, 1, picked
    x, k = mesh.jacobi(sch, x, om, mc.sweeps - 1, mc.eps)
    return x, 1 + k, picked
