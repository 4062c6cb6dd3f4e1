"""Two-point entropy-conservative flux for the vdW gas (oracle; test infrastructure only).

Sec. 3.1: with the parameter vector z = (rho, v, T) (eq. parameter_vector) the
Tadmor conditions (eq. ECCondition_comp)
    [[V]]^T U~ = [[phi]],   [[V]]^T F~_j = [[psi_j]]
are split into the jumps of z (eq. jumpV), the coefficients of equal jumps are
matched (eq. linear_U, linear_F) and the lower-triangular system is solved
(Theorem 3.1 and the explicit solution printed after it).

This module restates that solution in general units (a, b, R, c_v): the same
jump identities with R/{rho}^ln + R b/{1 - b rho}^ln + R b/Pi - 2a/{T} in place
of the reduced-unit determinant D.  ``ec_flux_units_b_1d`` is a direct
transcription of the paper's explicit reduced-unit formulas and serves as an
independent check of the restatement.
"""
import numpy as np


def mean(al, ar):
    """Arithmetic mean {a} = (a_l + a_r)/2 (Sec. 3.1)."""
    return 0.5 * (al + ar)


def log_mean(al, ar):
    """Logarithmic mean {a}^ln = [[a]] / [[ln a]] for a > 0 (Sec. 3.1, after eq. jumpV).

    With f = (a_l - a_r)/(a_l + a_r), [[ln a]] = 2 artanh(f), so
    {a}^ln = (a_l + a_r) / (2 F) with F = artanh(f)/f.  For |f| < 1e-2 the
    Taylor series F = sum_k f^(2k)/(2k+1) (six terms, remainder < 1e-24) is
    used; it also gives the limit {a}^ln = a at a_l = a_r.
    """
    al = np.asarray(al, dtype=np.float64)
    ar = np.asarray(ar, dtype=np.float64)
    f = (al - ar) / (al + ar)
    u = f * f
    small = np.abs(f) < 1e-2
    F_series = 1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0 + u * (1.0 / 9.0 + u / 11.0))))
    with np.errstate(divide="ignore", invalid="ignore"):
        F_exact = np.arctanh(f) / f
    F = np.where(small, F_series, F_exact)
    return (al + ar) / (2.0 * F)


def ec_determinant(g, rho_l, T_l, rho_r, T_r):
    """Coefficient of [[rho]] in [[V_1]] (eq. jumpV), general units.

    D = R/{rho}^ln + R b/{1 - b rho}^ln + R b/((1 - b rho_l)(1 - b rho_r)) - 2a/{T};
    Theorem 3.1 shows D > 0 under eq. mean_constraint.
    """
    Pi = (1.0 - g.b * rho_l) * (1.0 - g.b * rho_r)
    D = g.R / log_mean(rho_l, rho_r) - 2.0 * g.a / mean(T_l, T_r) + g.R * g.b / Pi
    if g.b > 0.0:
        D = D + g.R * g.b / log_mean(1.0 - g.b * rho_l, 1.0 - g.b * rho_r)
    return D


def ec_flux(g, rho_l, v_l, T_l, rho_r, v_r, T_r):
    """Two-point EC pair (U~, F~_j) in general units (Sec. 3.1, explicit solution).

    v_l, v_r have shape (d, ...).  Returns (Ut, Ft): Ut has shape (d+2, ...),
    Ft has shape (d, d+2, ...) with Ft[j] = F~_j.

    Matching the coefficients of [[rho]], [[v_m]] and [[T]]:
      D U~_1         = {rho}(R b/Pi - a/{T}) + {g}          with g = R/(1 - b rho) - a rho/T
      U~_{1+m}       = {v_m} U~_1
      {1/T} U~_E     = a {rho}{rho/T} - B0 U~_1 + sum_m {v_m/T} U~_{1+m}
      D F~_{j,1}     = {rho v_j}(R b/Pi - a/{T}) + {g}{v_j}
      F~_{j,1+m}     = {v_m} F~_{j,1} + delta_mj {rho}{T}{g}
      {1/T} F~_{j,E} = a {rho v_j}{rho/T} - B0 F~_{j,1} + sum_m {v_m/T} F~_{j,1+m}
    with B0 = sum_m {v_m^2/T}/2 - c_v {T}/{T}^ln + 2a {rho/T}.
    """
    d = v_l.shape[0]
    Pi = (1.0 - g.b * rho_l) * (1.0 - g.b * rho_r)
    D = ec_determinant(g, rho_l, T_l, rho_r, T_r)
    T_m = mean(T_l, T_r)
    rho_m = mean(rho_l, rho_r)
    g_l = g.R / (1.0 - g.b * rho_l) - g.a * rho_l / T_l
    g_r = g.R / (1.0 - g.b * rho_r) - g.a * rho_r / T_r
    g_m = mean(g_l, g_r)
    rhoT_m = mean(rho_l / T_l, rho_r / T_r)
    invT_m = mean(1.0 / T_l, 1.0 / T_r)
    coef = g.R * g.b / Pi - g.a / T_m
    B0 = (0.5 * sum(mean(v_l[m] ** 2 / T_l, v_r[m] ** 2 / T_r) for m in range(d))
          - g.cv * T_m / log_mean(T_l, T_r) + 2.0 * g.a * rhoT_m)
    vm = [mean(v_l[m], v_r[m]) for m in range(d)]
    vT = [mean(v_l[m] / T_l, v_r[m] / T_r) for m in range(d)]

    shape = np.broadcast(rho_l, rho_r).shape
    Ut = np.empty((d + 2,) + shape)
    Ut[0] = (rho_m * coef + g_m) / D
    for m in range(d):
        Ut[1 + m] = vm[m] * Ut[0]
    Ut[-1] = (g.a * rho_m * rhoT_m - B0 * Ut[0] + sum(vT[m] * Ut[1 + m] for m in range(d))) / invT_m

    Ft = np.empty((d, d + 2) + shape)
    for j in range(d):
        rv_m = mean(rho_l * v_l[j], rho_r * v_r[j])
        Ft[j, 0] = (rv_m * coef + g_m * vm[j]) / D
        for m in range(d):
            Ft[j, 1 + m] = vm[m] * Ft[j, 0]
        Ft[j, 1 + j] += rho_m * T_m * g_m
        Ft[j, -1] = (g.a * rv_m * rhoT_m - B0 * Ft[j, 0]
                     + sum(vT[m] * Ft[j, 1 + m] for m in range(d))) / invT_m
    return Ut, Ft


def ec_flux_units_b_1d(delta, z_l, z_r):
    """The paper's explicit U~ and F~_1 in reduced units, 1D (Sec. 3.1, after Theorem 3.1).

    z = (z1, z2, z5) = (rho, v_1, T).  In these units the momentum flux carries
    3p/8 (eq. Euler).  Written from the printed closed forms with d = 1 (the
    sums over m = 2..4 keep the single velocity component).
    """
    z1l, z2l, z5l = z_l
    z1r, z2r, z5r = z_r
    m1 = mean(z1l, z1r)
    m2 = mean(z2l, z2r)
    m5 = mean(z5l, z5r)
    prod3 = (3.0 - z1l) * (3.0 - z1r)
    D = 1.0 / log_mean(z1l, z1r) + 1.0 / log_mean(3.0 - z1l, 3.0 - z1r) + 3.0 / prod3 - 9.0 / (4.0 * m5)
    gmean = mean(-9.0 / 8.0 * z1l / z5l + 3.0 / (3.0 - z1l), -9.0 / 8.0 * z1r / z5r + 3.0 / (3.0 - z1r))
    z1_z5 = mean(z1l / z5l, z1r / z5r)
    z2sq_z5 = mean(z2l**2 / z5l, z2r**2 / z5r)
    z2_z5 = mean(z2l / z5l, z2r / z5r)
    inv_z5 = mean(1.0 / z5l, 1.0 / z5r)
    z1z2 = mean(z1l * z2l, z1r * z2r)
    lnz5 = log_mean(z5l, z5r)
    bracket = 0.5 * z2sq_z5 - m5 / (delta * lnz5) + 9.0 / 4.0 * z1_z5

    U1 = (m1 * (-9.0 / 8.0 / m5 + 3.0 / prod3) + gmean) / D
    U2 = m2 * U1
    U5 = (-bracket * U1 + z2_z5 * U2 + 9.0 / 8.0 * m1 * z1_z5) / inv_z5

    F1 = (z1z2 * (-9.0 / 8.0 / m5 + 3.0 / prod3) + gmean * m2) / D
    F2 = m1 * m5 * gmean + m2 * F1
    F5 = (-bracket * F1 + z2_z5 * F2 + 9.0 * z1z2 / 8.0 * z1_z5) / inv_z5
    return np.array([U1, U2, U5]), np.array([F1, F2, F5])
