"""Thermodynamics of the van der Waals gas (oracle; test infrastructure only).

General units: p = rho R T/(1 - b rho) - a rho^2, e = c_v T - a rho
(Sec. 1, eq. vdWEOS).  The paper's reduced units (Sec. 2, eq. nondimEOS) are
the same family with (a, b, R, c_v) = (9/8, 1/3, 1, 1/delta) and a flux
pressure of 3p/8; the units used by the workloads here keep a plain p in the
flux and take (a, b, R, c_v) = (3, 1/3, 8/3, (8/3)/delta).  a = b = 0 is the
ideal gas with gamma = 1 + R/c_v.

All arrays are float64.
"""
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Gas:
    """van der Waals constants (Sec. 1, eq. vdWEOS)."""
    a: float
    b: float
    R: float
    cv: float

    @property
    def delta(self):
        """delta = gamma - 1 = R / c_v (Sec. 1)."""
        return self.R / self.cv


def gas_units_a(delta=0.0125):
    """Reduced units with a plain-pressure flux: p = 8 rho T/(3 - rho) - 3 rho^2."""
    R = 8.0 / 3.0
    return Gas(a=3.0, b=1.0 / 3.0, R=R, cv=R / delta)


def gas_units_b(delta=0.0125):
    """The paper's reduced units (Sec. 2): flux pressure 3p/8 with p from eq. nondimEOS."""
    return Gas(a=9.0 / 8.0, b=1.0 / 3.0, R=1.0, cv=1.0 / delta)


def ideal_gas(gamma=1.4, R=1.0):
    """a = b = 0: the EOS reduces to the ideal gas law (Sec. 1)."""
    return Gas(a=0.0, b=0.0, R=R, cv=R / (gamma - 1.0))


# ---------------------------------------------------------------- EOS, Sec. 1

def pressure(g, rho, T):
    """eq. vdWEOS: p = rho R T / (1 - b rho) - a rho^2."""
    return rho * g.R * T / (1.0 - g.b * rho) - g.a * rho**2


def temperature(g, rho, p):
    """Inverse of eq. vdWEOS for T; the paper's z_5 in eq. parameter_vector."""
    return (p + g.a * rho**2) * (1.0 - g.b * rho) / (g.R * rho)


def internal_energy(g, rho, T):
    """eq. vdWEOS: e = c_v T - a rho."""
    return g.cv * T - g.a * rho


def sound_speed2(g, rho, T):
    """c_s^2 = (1 + delta) R T/(1 - b rho)^2 - 2 a rho (Sec. 1, after eq. fundamental)."""
    return (1.0 + g.delta) * g.R * T / (1.0 - g.b * rho) ** 2 - 2.0 * g.a * rho


def fundamental_derivative(g, rho, T):
    """G = nu^3/(2 c^2) (d^2 p/d nu^2)_s (Sec. 1, eq. fundamental).

    Along an isentrope of the vdW gas T (nu - b)^delta is constant (s above),
    so p(nu) = R K (nu - b)^(-1-delta) - a/nu^2 with K = T (nu - b)^delta and
    the second derivative is p_nunu = (1+delta)(2+delta) R T/(nu - b)^3 - 6 a/nu^4.
    """
    nu = 1.0 / rho
    p_nunu = (1.0 + g.delta) * (2.0 + g.delta) * g.R * T / (nu - g.b) ** 3 - 6.0 * g.a / nu**4
    return nu**3 * p_nunu / (2.0 * sound_speed2(g, rho, T))


def entropy(g, rho, T):
    """Specific entropy s = c_v ln T + R ln((1 - b rho)/rho) (Sec. 1; reduced form Sec. 2).

    The sign of the volume term follows the reduced form ln((3 - rho)/(2 rho))
    of Sec. 2 (the general form printed in Sec. 1 carries a sign slip); the
    additive constant is dropped because only jumps of V enter the scheme.
    """
    return g.cv * np.log(T) + g.R * np.log((1.0 - g.b * rho) / rho)


def admissible(g, rho, T):
    """eq. coefflimit / eq. Tlimit: 0 < rho < 1/b, T > a/(4Rb), R T - 2 a rho (1 - b rho)^2 > 0."""
    ok = rho > 0.0
    if g.b > 0.0:
        ok &= rho < 1.0 / g.b
        ok &= T > g.a / (4.0 * g.R * g.b)
    ok &= T > 0.0
    ok &= g.R * T - 2.0 * g.a * rho * (1.0 - g.b * rho) ** 2 > 0.0
    return ok


# ------------------------------------------------- conservative <-> primitive

def prim_to_cons(g, rho, v, p):
    """U = (rho, rho v, E) with E = rho e + rho |v|^2 / 2 (Sec. 1, eq. ConserLaw2).

    v has shape (d, ...).  Returns U with shape (d + 2, ...).
    """
    T = temperature(g, rho, p)
    E = rho * internal_energy(g, rho, T) + 0.5 * rho * np.sum(v**2, axis=0)
    return np.concatenate([rho[None], rho[None] * v, E[None]], axis=0)


def cons_to_prim(g, U):
    """Primitive (rho, v, T, p) from U: e = E/rho - |v|^2/2, T = (e + a rho)/c_v."""
    rho = U[0]
    v = U[1:-1] / rho
    e = U[-1] / rho - 0.5 * np.sum(v**2, axis=0)
    T = (e + g.a * rho) / g.cv
    p = pressure(g, rho, T)
    return rho, v, T, p


def flux(g, U, n):
    """Physical flux projected on a direction n: sum_j n_j F_j(U) (eq. ConserLaw3).

    n has shape (d, ...) (broadcast against U[0]).
    """
    rho, v, T, p = cons_to_prim(g, U)
    vn = np.sum(n * v, axis=0)
    out = np.empty(np.broadcast(U, vn[None]).shape, dtype=np.result_type(U, n))
    out[0] = rho * vn
    for m in range(v.shape[0]):
        out[1 + m] = rho * v[m] * vn + p * n[m]
    out[-1] = (U[-1] + p) * vn
    return out


# ----------------------------------------------- entropy pair, Def. 2.1

def entropy_function(g, U):
    """eta = -rho s (eq. van der WaalsEntropy)."""
    rho, v, T, p = cons_to_prim(g, U)
    return -rho * entropy(g, rho, T)


def entropy_variables(g, U):
    """V = eta'(U)^T (Sec. 2), written in general units.

    With eta = -rho s the derivative is V = ((e + p/rho)/T - s - |v|^2/(2T), v/T, -1/T);
    for the vdW gas (e + p/rho)/T = c_v - 2 a rho/T + R/(1 - b rho).
    """
    rho, v, T, p = cons_to_prim(g, U)
    s = entropy(g, rho, T)
    V1 = g.cv - s - 2.0 * g.a * rho / T + g.R / (1.0 - g.b * rho) - 0.5 * np.sum(v**2, axis=0) / T
    return np.concatenate([V1[None], v / T, (-1.0 / T)[None]], axis=0)


def potential(g, U):
    """phi = V^T U - eta = p/T (eq. van der WaalsPoten, general units)."""
    rho, v, T, p = cons_to_prim(g, U)
    return p / T


def flux_potential(g, U, j):
    """psi_j = V^T F_j - q_j = p v_j / T (eq. van der WaalsPoten, general units)."""
    rho, v, T, p = cons_to_prim(g, U)
    return p * v[j] / T


# ----------------------------------------------- Remark 2.2 (input helper)

def spinodal_densities(T):
    """Roots rho** (point N) and rho*** (point M) of p_nu = 0 for T0 < T < 1 (Remark 2.2, reduced units)."""
    th = np.arccos(2.0 * T - 1.0)
    rho_N = 2.0 * np.cos((th + 2.0 * np.pi) / 3.0) + 2.0
    rho_M = 2.0 * np.cos((th + 4.0 * np.pi) / 3.0) + 2.0
    return rho_N, rho_M
