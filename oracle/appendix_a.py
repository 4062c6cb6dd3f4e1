"""The alternative parameter vectors of Appendix A (oracle; test infrastructure only).

App. A shows why the choice of parameter vector matters for the explicit two-point EC flux.  For three other
vectors z it writes the jump of the entropy variables as a linear system [[V]] = M [[z]] (1D, the paper's reduced
units: a = 9/8, b = 1/3, R = 1, so 1 - b rho = (3 - rho)/3 and the EOS terms read 3/(3 - rho), 9 rho/(4 T)) and
prints the determinant of M.  The flux is explicit only where that determinant is nonzero; the appendix states
that each of the three can vanish for admissible states, unlike the vector of Sec. 3.1 under Theorem 3.1.

Notation: {a} is the arithmetic mean, {a}^ln the logarithmic mean, [[a]] = a_r - a_l; delta = gamma - 1.
Each function takes the two states (rho, v, T) and delta and returns (M, z_l, z_r, det) with M the 3 x 3 matrix
of coefficients (rows [[V_1]], [[V_2]], [[V_3]]; columns [[z_1]], [[z_2]], [[z_3]]) and det the appendix's closed
form of its determinant (for the first vector with the factor the printed form drops, see vector_1).
"""
import numpy as np

from .ecflux import log_mean


def _mean(a, b):
    return 0.5 * (a + b)


def vector_1(l, r, delta):
    """z = ((3 - rho)/T, T/(3 - rho)^2, v): with A = {z1}{z2} + {z1 z2} and B = {z1}^2, [[1/T]] = A[[z1]] + B[[z2]]
    (z1^2 z2 = 1/T), and [[-s]] = [[1/T]]/(delta {1/T}^ln) + 3 [[z1 z2]]/{3 z1 z2 - 1}^ln."""
    def z(s):
        rho, v, T = s
        return np.array([(3.0 - rho) / T, T / (3.0 - rho) ** 2, v])
    zl, zr = z(l), z(r)
    m = _mean(zl, zr)
    z1z2 = _mean(zl[0] * zl[1], zr[0] * zr[1])
    A = m[0] * m[1] + z1z2
    B = m[0] ** 2
    iT_ln = log_mean(zl[0] ** 2 * zl[1], zr[0] ** 2 * zr[1])
    iT = _mean(zl[0] ** 2 * zl[1], zr[0] ** 2 * zr[1])
    q_ln = log_mean(3.0 * zl[0] * zl[1] - 1.0, 3.0 * zr[0] * zr[1] - 1.0)
    z3sq = _mean(zl[2] ** 2, zr[2] ** 2)
    M = np.array([
        [A / (delta * iT_ln) + 3.0 * m[1] / q_ln + 3.0 * m[1] - 6.75 * A - 0.5 * z3sq * A + 2.25,
         B / (delta * iT_ln) + 3.0 * m[0] / q_ln + 3.0 * m[0] - 6.75 * B - 0.5 * z3sq * B,
         -iT * m[2]],
        [m[2] * A, m[2] * B, iT],
        [-A, -B, 0.0]])
    # det M = {1/T} (B M_11 - A M_12): the paper prints 3/4 where the expansion gives (3/4) B
    det = 3.0 * iT * ((B * m[1] - A * m[0]) / q_ln + B * m[1] - A * m[0] + 0.75 * B)
    return M, zl, zr, det


def vector_2(l, r, delta):
    """z = (rho, 1/T, v)."""
    def z(s):
        rho, v, T = s
        return np.array([rho, 1.0 / T, v])
    zl, zr = z(l), z(r)
    m = _mean(zl, zr)
    z3sq = _mean(zl[2] ** 2, zr[2] ** 2)
    K = (1.0 / log_mean(zl[0], zr[0]) + 1.0 / log_mean(3.0 - zl[0], 3.0 - zr[0])
         + 3.0 / ((3.0 - zl[0]) * (3.0 - zr[0])) - 2.25 * m[1])
    M = np.array([
        [K, 1.0 / (delta * log_mean(zl[1], zr[1])) - 2.25 * m[0] - 0.5 * z3sq, -m[1] * m[2]],
        [0.0, m[2], m[1]],
        [0.0, -1.0, 0.0]])
    det = m[1] * K
    return M, zl, zr, det


def vector_3(l, r, delta):
    """z = (-9/(8T) + 1/(3 - rho), 1/(3 - rho), v): [[1/T]] = (8/9)[[z2]] - (8/9)[[z1]] =: A[[z1]] + B[[z2]]."""
    def z(s):
        rho, v, T = s
        return np.array([-9.0 / (8.0 * T) + 1.0 / (3.0 - rho), 1.0 / (3.0 - rho), v])
    zl, zr = z(l), z(r)
    m = _mean(zl, zr)
    A, B = -8.0 / 9.0, 8.0 / 9.0
    iT = _mean(1.0 / l[2], 1.0 / r[2])
    iT_ln = log_mean(1.0 / l[2], 1.0 / r[2])
    two_z2 = _mean(2.0 / zl[1], 2.0 / zr[1])
    q_ln = log_mean(l[0] / (3.0 - l[0]), r[0] / (3.0 - r[0]))
    z3sq = _mean(zl[2] ** 2, zr[2] ** 2)
    M = np.array([
        [A / (delta * iT_ln) + 6.0 - two_z2 - 0.5 * z3sq * A,
         B / (delta * iT_ln) - 3.0 + 3.0 / q_ln + m[0] / m[1] * two_z2 - 0.5 * z3sq * B,
         -iT * m[2]],
        [m[2] * A, m[2] * B, iT],
        [-A, -B, 0.0]])
    det = 8.0 / 9.0 * iT * (3.0 - two_z2 + 3.0 / q_ln + m[0] / m[1] * two_z2)
    return M, zl, zr, det


def theorem_3_1_D(l, r):
    """D of Theorem 3.1 (the parameter vector of Sec. 3.1, z_1 = rho, z_5 = T):
    D = 1/{rho}^ln + 1/{3 - rho}^ln + 3/((3 - rho_l)(3 - rho_r)) - 9/(4 {T})."""
    return (1.0 / log_mean(l[0], r[0]) + 1.0 / log_mean(3.0 - l[0], 3.0 - r[0])
            + 3.0 / ((3.0 - l[0]) * (3.0 - r[0])) - 9.0 / (4.0 * _mean(l[2], r[2])))
