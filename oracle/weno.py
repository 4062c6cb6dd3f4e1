"""Fifth-order multi-resolution WENO reconstruction (oracle; test infrastructure only).

Sec. 3.3 applies the fifth-order multi-resolution WENO reconstruction of its
reference [Wang et al. 2021] to the scaled entropy variables, with linear
weights lambda_0 = 0.95, lambda_1 = 0.045, lambda_2 = 0.005 (Sec. 5).  The
reference itself is not reproduced in the paper, so this module restates the
published multi-resolution WENO framework (Zhu & Shu, J. Comput. Phys. 2018)
in its finite-difference form, where the point values play the role of cell
averages:

  nested central stencils {i}, {i-1, i, i+1}, {i-2, ..., i+2};
  q_l = the polynomial of degree 0, 2, 4 matching those averages;
  p_1 = q_1, p_2 = (q_2 - g_12 p_1)/g_22, p_3 = (q_3 - g_13 p_1 - g_23 p_2)/g_33
        with g_lk = gamma_l / sum_{l' <= k} gamma_l';
  beta_2, beta_3 = sum_alpha int_I dx^(2 alpha - 1) (d^alpha q_l / dx^alpha)^2 dx
        (computed here from that definition by exact polynomial integration);
  beta_1 = min((w_i - w_{i-1})^2, (w_{i+1} - w_i)^2);
  tau = ((|beta_3 - beta_1| + |beta_3 - beta_2|)/2)^2;
  w~_l = gamma_l (1 + tau/(beta_l + eps)), normalised;  value = sum_l w_l p_l.

Reading of the weights (the paper lists lambda_0..2 without naming the
stencils): the dominant 0.95 goes to the 5-point stencil, 0.045 to the
3-point and 0.005 to the 1-point stencil.  eps = 1e-6 (Jiang and Shu's value;
the paper gives none).  The acoustic components of W = R^T T V for a smooth
entropy wave are flat at the face (R's face state makes R^T dV/dx vanish
there), so W_{i+1} = W_i to second order and beta_1 falls to O(h^6) while
beta_3 is O(h^4); with eps far below beta_3 the weights then drift to the
1-point value and the reconstruction loses orders until the mesh is fine.
With linear weights 1/3 each (Example 5.6) a 1e-12 eps left the 2D
operator at order 2 to 3 up to 128^2; with 1e-6 it reaches fifth order from
about 64^2.  Parity of the nonlinear weights is
unpinned: the cited paper is not available; the pins are the linear limit,
exactness on constants and the design order.
"""
from fractions import Fraction

import numpy as np
from numpy.polynomial import polynomial as P

# stencil offsets relative to node i of the three nested stencils
_STENCILS = ((0,), (-1, 0, 1), (-2, -1, 0, 1, 2))


def _average_matching_polynomial(offsets):
    """Coefficient map: values on cells -> monomial coefficients in x (unit cells, cell i = [-1/2, 1/2]).

    Returns M with coef = M @ w such that (1/1) int_{j-1/2}^{j+1/2} q(x) dx = w_j
    for every offset j.  Solved with exact rationals.
    """
    n = len(offsets)
    A = []
    for j in offsets:
        row = []
        for k in range(n):  # int x^k over [j-1/2, j+1/2]
            hi = Fraction(2 * j + 1, 2) ** (k + 1)
            lo = Fraction(2 * j - 1, 2) ** (k + 1)
            row.append((hi - lo) / (k + 1))
        A.append(row)
    # Gauss-Jordan on rationals
    M = [[Fraction(int(r == c)) for c in range(n)] for r in range(n)]
    A = [row[:] for row in A]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        M[col], M[piv] = M[piv], M[col]
        inv = 1 / A[col][col]
        A[col] = [x * inv for x in A[col]]
        M[col] = [x * inv for x in M[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
    return M  # coef_k = sum_j M[k][j] w_j


def interface_weights(offsets):
    """Values of the matching polynomial at x_{i+1/2}: list of rational weights on w_j."""
    M = _average_matching_polynomial(offsets)
    n = len(offsets)
    half = Fraction(1, 2)
    return [sum(M[k][j] * half**k for k in range(n)) for j in range(n)]


def smoothness_matrix(offsets):
    """Quadratic form B with beta = w^T B w, from the Jiang-Shu definition on cell i.

    beta = sum_{alpha=1}^{deg} int_{-1/2}^{1/2} (d^alpha q/dx^alpha)^2 dx
    (unit spacing, so the dx^(2 alpha - 1) factors are 1).
    """
    M = np.array([[float(x) for x in row] for row in _average_matching_polynomial(offsets)])
    n = len(offsets)
    B = np.zeros((n, n))
    for a_idx in range(n):
        for b_idx in range(n):
            ea = np.zeros(n)
            ea[a_idx] = 1.0
            eb = np.zeros(n)
            eb[b_idx] = 1.0
            qa = M @ ea
            qb = M @ eb
            tot = 0.0
            for alpha in range(1, n):
                da = P.polyder(qa, alpha)
                db = P.polyder(qb, alpha)
                prod = P.polymul(da, db)
                anti = P.polyint(prod)
                tot += P.polyval(0.5, anti) - P.polyval(-0.5, anti)
            B[a_idx, b_idx] = tot
    return B


_Q2 = np.array([float(x) for x in interface_weights(_STENCILS[1])])   # (-1, 5, 2)/6
_Q3 = np.array([float(x) for x in interface_weights(_STENCILS[2])])   # (2, -13, 47, 27, -3)/60
_B2 = smoothness_matrix(_STENCILS[1])
_B3 = smoothness_matrix(_STENCILS[2])


def mr_weno5(w, gammas=(0.005, 0.045, 0.95), eps=1e-6):
    """Reconstruct the value at x_{i+1/2} from w = (w_{i-2}, ..., w_{i+2}) (leading axis of length 5).

    gammas = (1-point, 3-point, 5-point) linear weights.
    """
    w = np.asarray(w, dtype=np.float64)
    g1, g2, g3 = gammas
    q1 = w[2]
    q2 = np.tensordot(_Q2, w[1:4], axes=1)
    q3 = np.tensordot(_Q3, w, axes=1)
    g12 = g1 / (g1 + g2)
    g22 = g2 / (g1 + g2)
    p1 = q1
    p2 = (q2 - g12 * p1) / g22
    p3 = (q3 - g1 * p1 - g2 * p2) / g3
    beta1 = np.minimum((w[2] - w[1]) ** 2, (w[3] - w[2]) ** 2)
    # beta integrates squared derivatives of the polynomial, so it ignores a constant added to
    # the data (B 1 = 0): the forms are evaluated on w - w_i, which keeps rounding of |w|^2-sized
    # terms out of indicators that can be far smaller (data with a large mean and a small variation)
    d = w - w[2]
    beta2 = np.einsum("a...,ab,b...->...", d[1:4], _B2, d[1:4])
    beta3 = np.einsum("a...,ab,b...->...", d, _B3, d)
    tau = (0.5 * (np.abs(beta3 - beta1) + np.abs(beta3 - beta2))) ** 2
    wt1 = g1 * (1.0 + tau / (beta1 + eps))
    wt2 = g2 * (1.0 + tau / (beta2 + eps))
    wt3 = g3 * (1.0 + tau / (beta3 + eps))
    s = wt1 + wt2 + wt3
    return (wt1 * p1 + wt2 * p2 + wt3 * p3) / s
