"""Time step, SSP-RK3 and one full moving-mesh step (oracle; test infrastructure only).

Sec. 5 (eq. cfl) fixes Delta t_n from the spectral radii; the SSP-RK3 of
Gottlieb, Shu & Tadmor (cited in Sec. 1 and Sec. 5) integrates (JU, J);
Sec. 4 moves the mesh once per step with velocity xdot = Delta_gamma dx / Delta t_n.

Readings of points the paper leaves open:
  * eq. cfl takes the spectral radius at t_n, which contains the mesh velocity
    xdot^n = Delta_gamma dx / Delta t_n (Sec. 4), so the two define each other.
    Delta t^(0) from the current mesh with xdot = 0 gives xdot; then
    Delta t_n = min(Delta t^(0), CFL / max_i sum_k rho_{i,k}(xdot) / dxi_k) with
    that xdot.  The mesh moves by xdot Delta t_n = Delta_gamma' dx with
    Delta_gamma' = Delta_gamma Delta t_n / Delta t^(0) <= Delta_gamma, which still
    meets the bounds that define Delta_gamma, so eq. cfl and those bounds both hold;
  * the mesh moves with constant xdot over the step; RK stage s evaluates the
    operator on x^(s) = x^n + c_s Delta t xdot with c = (0, 1, 1/2) (the
    stage times of SSP-RK3) and recomputes the metrics there, which keeps the
    discrete SCL at every stage;
  * J is advanced only by the discrete VCL (eq. semi_J) after its initial
    value from the metrics;
  * the last step is shortened to reach t_end exactly.
"""
from dataclasses import dataclass

import numpy as np

from . import mesh, thermo
from .operator import axis_of, direction_metrics, rhs

# Shu-Osher form of SSP-RK3: U^(s+1) = a_s U^n + b_s (U^(s) + dt L(U^(s)))
RK3_A = (0.0, 0.75, 1.0 / 3.0)
RK3_B = (1.0, 0.25, 2.0 / 3.0)
RK3_C = (0.0, 1.0, 0.5)          # stage times as fractions of dt


@dataclass
class MeshControl:
    """Mesh redistribution parameters (Sec. 4, Sec. 5)."""
    moving: bool = False
    monitor: str = "vdw"           # "vdw": eq. van der Waalsmonitor; "smooth": eq. van der Waalssinmonitor
    alphas: tuple = (1200.0, 1200.0, 1200.0)
    kappa: int = 2                 # delta_1 = rho, delta_2 = G (vdw monitor)
    filter_passes: int = 5
    sweeps: int = 5                # mu
    eps: float = 0.0


def cfl_dt(sch, JU, J, x, cfl, xdot=None):
    """eq. cfl: Delta t = CFL / max_i sum_k rho_{i,k} / dxi_k with the spectral radius of the
    xi_k-direction flux Jacobian, rho_{i,k} = (|J xi_{k,t} + n_k . v| + L_k c) / J, where
    J xi_{k,t} = -xdot . n_k (eq. VCLCoeff); xdot = None is a mesh at rest."""
    g = sch.gas
    U = JU / J
    rho, v, T, p = thermo.cons_to_prim(g, U)
    c = np.sqrt(thermo.sound_speed2(g, rho, T))
    tot = np.zeros_like(J)
    xd = np.zeros_like(x) if xdot is None else xdot
    for k in range(sch.dim):
        n, xt = direction_metrics(sch, x, xd, k, 0)
        L = np.sqrt(np.sum(n**2, axis=0))
        vn = np.sum(n * v, axis=0)
        tot += (np.abs(xt + vn) + L * c) / J / sch.dxi[k]
    return cfl / float(np.max(tot))


def redistribute(sch, mc, JU, J, x, dt):
    """Sec. 4: monitor -> filter -> Jacobi -> limiter -> xdot.  Returns (xdot, sweeps, Delta_gamma)."""
    g = sch.gas
    U = JU / J
    rho, v, T, p = thermo.cons_to_prim(g, U)
    if mc.monitor == "smooth":
        om = mesh.monitor_smooth(rho, mc.alphas, sch.dim, sch.bc, sch.dxi)
    else:
        G = thermo.fundamental_derivative(g, rho, T)
        fields = [rho, G][:mc.kappa]
        om = mesh.monitor_vdw(fields, G, mc.alphas, sch.dim, sch.bc, sch.dxi)
    for _ in range(mc.filter_passes):
        om = mesh.low_pass(om, sch.dim, sch.bc)
    xit, sweeps = mesh.jacobi(sch, x, om, mc.sweeps, mc.eps)
    dx = xit - x
    gam = mesh.limiter(sch, x, dx)
    return gam * dx / dt, sweeps, gam


def rk_stage(sch, s, dt, JUn, Jn, JUs, Js, xn, xdot):
    """SSP-RK3 stage s (0, 1, 2) on (JU, J) with the operator on the stage mesh."""
    xs = xn + RK3_C[s] * dt * xdot
    dU, dJ = rhs(sch, JUs, Js, xs, xdot)
    a, b = RK3_A[s], RK3_B[s]
    return a * JUn + b * (JUs + dt * dU), a * Jn + b * (Js + dt * dJ)


def step(sch, mc, JU, J, x, t, t_end, cfl, dt_fixed=None):
    """One full step: Delta t, mesh velocity, three RK stages, mesh update.

    Returns (JU, J, x, t, info) with info = dict(dt, sweeps, gamma).
    """
    dt = dt_fixed if dt_fixed is not None else cfl_dt(sch, JU, J, x, cfl)
    dt = min(dt, t_end - t)
    if mc.moving:
        xdot, sweeps, gam = redistribute(sch, mc, JU, J, x, dt)
        if dt_fixed is None:
            dt = min(dt, cfl_dt(sch, JU, J, x, cfl, xdot))
    else:
        xdot, sweeps, gam = np.zeros_like(x), 0, 0.0
    JU1, J1 = rk_stage(sch, 0, dt, JU, J, JU, J, x, xdot)
    JU2, J2 = rk_stage(sch, 1, dt, JU, J, JU1, J1, x, xdot)
    JU3, J3 = rk_stage(sch, 2, dt, JU, J, JU2, J2, x, xdot)
    return JU3, J3, x + dt * xdot, t + dt, dict(dt=dt, sweeps=sweeps, gamma=gam)


def run(sch, mc, JU, J, x, t_end, cfl, dt_fixed=None, max_steps=10**7):
    """Advance to t_end; returns (JU, J, x, steps)."""
    t = 0.0
    nsteps = 0
    while t < t_end * (1.0 - 1e-14) and nsteps < max_steps:
        JU, J, x, t, _ = step(sch, mc, JU, J, x, t, t_end, cfl, dt_fixed)
        nsteps += 1
    return JU, J, x, nsteps
