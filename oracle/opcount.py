"""Operation count of one RK stage (operator and Shu-Osher combination), from the oracle itself (test
infrastructure only).

The roofline of the ALU-bound stage kernels needs the algorithmic work per node and stage.  This module counts it by
running the oracle's stage on arrays that tally every elementwise floating-point operation they take part in:
+, -, *, / and square roots, logarithms and the other transcendental functions count one per element (a fused
multiply-add would count two); selections, comparisons, absolute values, signs, maxima and minima count nothing.
Tensor contractions (the eigen-projections, the reconstruction's coefficient maps) count one multiply and one add
per term.  Two corrections turn the oracle's count into the algorithm's:
  * the oracle evaluates each pair flux F(U_i, U_{i+m}) once for every face that uses it (m faces), the algorithm
    once: the operations inside the pair fluxes are divided by the mean reuse (w + 1)/2 = 2 for w = 3;
  * the oracle also evaluates node quantities and pair fluxes on the ghost nodes of each line: the count is taken
    on periodic meshes of three sizes, and the leading coefficient of the fit (linear in the node count in 1D,
    quadratic in n on n x n meshes in 2D) is the per-node count.
The oracle's logarithmic mean evaluates both its series and its artanh branch for every pair (np.where); that
adds a few operations per mean, under 1% of the total, and is left in.
Run ``python -m oracle.opcount`` to print the counts.
"""
import contextlib

import numpy as np

from . import ecflux, mesh, operator, stepper, thermo, weno

# ufuncs that count one operation per output element
_ARITH = {"add", "subtract", "multiply", "divide", "true_divide", "sqrt", "log", "log1p", "exp", "power",
          "arctanh", "arctan2", "reciprocal", "square", "cos", "sin", "arccos"}


class _Tally:
    def __init__(self):
        self.total = 0
        self.pair = 0
        self.in_pair = False

    def add(self, n):
        self.total += n
        if self.in_pair:
            self.pair += n


_TALLY = None


def _unwrap(x):
    if isinstance(x, Counted):
        return x.view(np.ndarray)
    if isinstance(x, (list, tuple)):
        return type(x)(_unwrap(y) for y in x)
    if isinstance(x, dict):
        return {k: _unwrap(v) for k, v in x.items()}
    return x


def _wrap(x):
    if isinstance(x, np.ndarray) and not isinstance(x, Counted) and x.dtype.kind == "f":
        return x.view(Counted)
    if isinstance(x, tuple):
        return tuple(_wrap(y) for y in x)
    if isinstance(x, list):
        return [_wrap(y) for y in x]
    return x


def _einsum_terms(spec, ops):
    """Number of multiply-add terms of an einsum: the product of the extents of all its indices."""
    lhs = spec.split("->")[0].split(",")
    sizes, ell = {}, []
    for sub, o in zip(lhs, ops):
        shape = np.shape(o)
        if "..." in sub:
            pre, post = sub.split("...")
            n_ell = len(shape) - len(pre) - len(post)
            ell.append(shape[len(pre):len(pre) + n_ell])
            named = list(zip(pre, shape[:len(pre)])) + list(zip(post, shape[len(shape) - len(post):]))
        else:
            named = list(zip(sub, shape))
        for ch, n in named:
            sizes[ch] = max(sizes.get(ch, 1), n)
    ell_size = int(np.prod(np.broadcast_shapes(*ell))) if ell else 1
    return int(np.prod(list(sizes.values()) or [1])) * ell_size


class Counted(np.ndarray):
    """An ndarray whose elementwise arithmetic is tallied."""

    def __array_ufunc__(self, ufunc, method, *inputs, **kwargs):
        result = getattr(ufunc, method)(*_unwrap(inputs), **_unwrap(kwargs))
        if _TALLY is not None and ufunc.__name__ in _ARITH:
            if method == "__call__":
                _TALLY.add(int(np.size(result[0] if isinstance(result, tuple) else result)))
            elif method == "reduce":
                _TALLY.add(int(np.size(_unwrap(inputs[0])) - np.size(result)))
        return _wrap(result)

    def __array_function__(self, func, types, args, kwargs):
        pargs, pkw = _unwrap(args), _unwrap(kwargs)
        result = func(*pargs, **pkw)
        if _TALLY is not None:
            if func is np.einsum:
                _TALLY.add(2 * _einsum_terms(pargs[0], pargs[1:]))
            elif func is np.tensordot:
                axes = pkw.get("axes", pargs[2] if len(pargs) > 2 else 2)
                a = pargs[0]
                k = np.shape(a)[-1] if axes == 1 else int(np.prod(np.shape(a)[-axes:]))
                _TALLY.add(2 * k * int(np.size(result)))
        return _wrap(result)


class _NumpyShim:
    """numpy as the oracle modules see it while counting: asarray keeps the tallying subclass."""

    def __getattr__(self, name):
        return getattr(np, name)

    @staticmethod
    def asarray(a, dtype=None, **kw):
        return np.asanyarray(a, dtype=dtype, **kw)


@contextlib.contextmanager
def _counting():
    global _TALLY
    _TALLY = _Tally()
    modules = (ecflux, mesh, operator, stepper, thermo, weno)
    real_pair = operator.ec_flux

    def pair(*args, **kw):
        prev, _TALLY.in_pair = _TALLY.in_pair, True
        try:
            return real_pair(*args, **kw)
        finally:
            _TALLY.in_pair = prev

    for m in modules:
        m.np = _NumpyShim()
    operator.ec_flux = pair
    try:
        yield _TALLY
    finally:
        for m in modules:
            m.np = np
        operator.ec_flux = real_pair
        _TALLY = None


def _stage_ops(dim, n, w=3):
    """Operations of one RK stage on an n (1D) or n x n (2D) periodic sine state on a moving mesh, with the pair
    fluxes' operations divided by their reuse (w + 1)/2."""
    g = thermo.gas_units_a()
    xs = np.arange(n) / n
    if dim == 1:
        x = xs[None].copy()
        rho = 0.5 + 0.2 * np.sin(2 * np.pi * xs)
        v = np.ones((1, n))
        p = np.ones(n)
    else:
        X, Y = np.meshgrid(xs, xs)
        x = np.stack([X, Y])
        rho = 0.5 + 0.2 * np.sin(2 * np.pi * (X + Y))
        v = np.stack([0.5 + 0 * X, 0.5 + 0 * X])
        p = np.ones_like(X)
    sch = operator.Scheme(gas=g, dim=dim, bc=("periodic",) * dim, dxi=(1.0 / n,) * dim, period=(1.0,) * dim, w=w)
    J = operator.node_jacobian(sch, x)
    JU = thermo.prim_to_cons(g, rho, v, p) * J
    xdot = 0.01 * np.ones_like(x)                       # a moving mesh: the metrics' mesh-velocity terms count
    c = [a.view(Counted) for a in (JU, J, x, xdot)]
    with _counting() as tally:
        stepper.rk_stage(sch, 1, 1e-4, c[0], c[1], c[0], c[1], c[2], c[3])
    reuse = (w + 1) / 2.0
    return tally.total - tally.pair + tally.pair / reuse, tally.pair / reuse


def per_node_stage(dim):
    """(operations, of which in pair fluxes) per node and RK stage, asymptotic in the mesh size."""
    if dim == 1:
        sizes = (128, 256)
        tot, pair = zip(*[_stage_ops(1, n) for n in sizes])
        return (tot[1] - tot[0]) / (sizes[1] - sizes[0]), (pair[1] - pair[0]) / (sizes[1] - sizes[0])
    sizes = (16, 24, 32)
    tot, pair = zip(*[_stage_ops(2, n) for n in sizes])
    A = np.array([[n * n, n, 1.0] for n in sizes])
    return float(np.linalg.solve(A, np.array(tot))[0]), float(np.linalg.solve(A, np.array(pair))[0])


if __name__ == "__main__":
    for d in (1, 2):
        a, ap = per_node_stage(d)
        print(f"dim {d}: {a:.0f} operations per node and RK stage ({ap:.0f} in the pair fluxes)")
