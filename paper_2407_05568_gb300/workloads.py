"""Seeded synthetic inputs: primitive fields (rho, v, p), meshes and run settings.

This module holds input recipes only -- no arithmetic of the numerical method.
Both the CUDA path and the oracle receive the same arrays from here and each
converts them to conservative variables with its own EOS.

Recipes follow the paper's test problems (Sec. 5): sine waves (Examples 5.1,
5.3), Riemann problems with the Table 5.1 states, and seeded four-quadrant /
shock-tube states near the critical point for the larger runs.  Units: the
reduced van der Waals units with a plain-pressure flux,
a = 3, b = 1/3, R = 8/3, c_v = R/0.0125, where p = 8 rho T/(3 - rho) - 3 rho^2.
"""
import numpy as np

UNITS_A = dict(a=3.0, b=1.0 / 3.0, R=8.0 / 3.0, cv=(8.0 / 3.0) / 0.0125)
IDEAL_14 = dict(a=0.0, b=0.0, R=1.0, cv=1.0 / 0.4)
VORTEX_BOX = 20.0      # side of the periodic box of the isentropic vortex (see isentropic_vortex)

# Table 5.1 (Example 5.2): (rho_l, v_l, p_l, rho_r, v_r, p_r)
TABLE_5_1 = {
    "RP1": (1.818, 0.0, 3.000, 0.275, 0.0, 0.575),
    "RP2": (0.879, 0.0, 1.090, 0.562, 0.0, 0.885),
    "RP3": (0.879, 0.0, 1.090, 0.275, 0.0, 0.575),
}

# Example 5.2's final times, printed as 0.15, 0.45 and 0.2 times Z_c^(-1/2) in the paper's reduced
# units (Z_c = p_c/(rho_c R T_c) = 3/8 for the van der Waals gas).  Those units carry a flux pressure
# 3p/8, so their velocities are sqrt(3/8) times the ones here and their times sqrt(8/3) times
# longer: t = sqrt(3/8) * 0.15 Z_c^(-1/2) = 0.15 in these units.
EXAMPLE_5_2_T_END = {"RP1": 0.15, "RP2": 0.45, "RP3": 0.2}


def _recipe_temperature(rho, p):
    """Acceptance test of the sampling recipe in the units above (input filter only)."""
    return (p + 3.0 * rho**2) * (3.0 - rho) / (8.0 * rho)


def _recipe_ok(rho, p, t_min=1.02):
    """Recipe acceptance region: 0 < rho < 3 and a supercritical temperature T >= t_min
    (T_c = 1).  Subcritical states can expand into the unstable region where
    4T - rho (3 - rho)^2 < 0; the states near the critical point with G < 0 lie just
    above T_c, so the recipe keeps them."""
    T = _recipe_temperature(rho, p)
    return (0.0 < rho < 3.0) and T >= t_min and 4.0 * T - rho * (3.0 - rho) ** 2 > 0.0


def _pair_ok(s1, s2):
    """Recipe acceptance between two neighbouring states: 4{T} - {rho}(3 - {rho})^2 > 0."""
    rm = 0.5 * (s1[0] + s2[0])
    Tm = 0.5 * (_recipe_temperature(s1[0], s1[-1]) + _recipe_temperature(s2[0], s2[-1]))
    return 4.0 * Tm - rm * (3.0 - rm) ** 2 > 0.0

# Table 5.2 (Example 5.4, Mach reflection): gamma, rho_l, v1_l, v2_l, p_l, rho_r, v1_r, v2_r, p_r in the
# paper's reduced units, and the incidence angle theta (degrees) of each case
TABLE_5_2 = {
    "P1": (1.4, 0.033, 5.016, 0.0, 3.001, 0.0156, 0.0, 0.0, 1.0),
    "D1": (1.0125, 0.629, -0.135, 0.0, 0.983, 0.879, 0.0, 0.0, 1.09),
}
MACH_THETA = {"P1": 20.0, "D1": 30.0}


def uniform_nodes(n, lo, hi, periodic):
    """Node coordinates and spacing: periodic -> n nodes on [lo, hi); else n nodes on [lo, hi]."""
    if periodic:
        d = (hi - lo) / n
        return lo + d * np.arange(n), d
    d = (hi - lo) / (n - 1)
    return lo + d * np.arange(n), d


def sine_1d(n=200, t_end=0.1, cfl=0.4, moving=False):
    """1D periodic density sine wave (Example 5.1 setup): rho = 0.5 + 0.2 sin(2 pi x), v = 1, p = 1
    on [0, 1); exact rho(x - t).  moving: Example 5.1's MM (the smooth-test monitor with
    alpha = (20, 15), 20 filter passes, 10 Jacobi sweeps); otherwise the fixed uniform mesh."""
    x, d = uniform_nodes(n, 0.0, 1.0, True)
    w = dict(gas=UNITS_A, dim=1, n=(n,), dxi=(d,), bc=("periodic",), period=(1.0,),
             x=x[None].copy(), rho=0.5 + 0.2 * np.sin(2 * np.pi * x), v=np.ones((1, n)),
             p=np.ones(n), t_end=t_end, cfl=cfl, moving=moving)
    if moving:
        w["mesh"] = dict(monitor="smooth", alphas=(20.0, 15.0), kappa=2, filter_passes=20, sweeps=10, eps=0.0)
    return w


def sine_2d(n=1024, t_end=0.1, cfl=0.4):
    """2D periodic sine wave (Example 5.3 setup): rho = 0.5 + 0.2 sin(2 pi (x + y)), v = (0.5, 0.5), p = 1."""
    x1, d = uniform_nodes(n, 0.0, 1.0, True)
    X, Yc = np.meshgrid(x1, x1)          # shape (n2, n1), X varies along the last axis
    return dict(gas=UNITS_A, dim=2, n=(n, n), dxi=(d, d), bc=("periodic", "periodic"),
                period=(1.0, 1.0), x=np.stack([X, Yc]),
                rho=0.5 + 0.2 * np.sin(2 * np.pi * (X + Yc)),
                v=np.stack([0.5 * np.ones_like(X), 0.5 * np.ones_like(X)]),
                p=np.ones_like(X), t_end=t_end, cfl=cfl, moving=False)


def sine_3d(n=64, t_end=0.1, cfl=0.3, moving=False):
    """3D periodic sine wave (Example 5.6 setup): rho = 0.5 + 0.2 sin(2 pi (x_1 + x_2 + x_3)),
    v = (0.3, 0.3, 0.3), p = 1 on [0, 1)^3; exact rho at (x - 0.3 t).  MM: the monitor of
    Example 5.1 (alpha = (20, 15), 20 filter passes), 10 Jacobi sweeps; MR-WENO linear weights
    1/3 each; CFL 0.3, the paper's choice in 3D (Sec. 5)."""
    x1, d = uniform_nodes(n, 0.0, 1.0, True)
    Z, Yc, X = np.meshgrid(x1, x1, x1, indexing="ij")      # shape (n3, n2, n1), x_1 along the last axis
    return dict(gas=UNITS_A, dim=3, n=(n, n, n), dxi=(d, d, d), bc=("periodic",) * 3,
                period=(1.0, 1.0, 1.0), x=np.stack([X, Yc, Z]),
                rho=0.5 + 0.2 * np.sin(2 * np.pi * (X + Yc + Z)),
                v=np.stack([0.3 * np.ones_like(X)] * 3), p=np.ones_like(X), t_end=t_end, cfl=cfl,
                moving=moving, weno_gammas=(1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0),
                mesh=dict(monitor="smooth", alphas=(20.0, 15.0), kappa=2, filter_passes=20, sweeps=10,
                          eps=0.0))


def spherical_shock_3d(n=64, t_end=None, cfl=0.3, moving=True):
    """3D spherically symmetric shock tube (Example 5.7 setup): the RP1 states of Table 5.1,
    (1.818, 0, 3.0) inside r < 0.5 and (0.275, 0, 0.575) outside, on the octant [0, 1]^3 with
    symmetry planes through the centre (x_k = 0) and outflow at x_k = 1; MM monitor with rho and
    G, alpha = (1200, 1200, 0) (Example 5.5's), 5 filter passes, 10 Jacobi sweeps; CFL 0.3 (the
    paper's in 3D).  The default final time is the example's t = 0.2 in the paper's reduced
    units, sqrt(3/8) 0.2 here (the conversion of EXAMPLE_5_2_T_END)."""
    t_end = 0.2 * np.sqrt(3.0 / 8.0) if t_end is None else t_end
    x1, d = uniform_nodes(n, 0.0, 1.0, False)
    Z, Yc, X = np.meshgrid(x1, x1, x1, indexing="ij")
    inside = X**2 + Yc**2 + Z**2 < 0.25
    return dict(gas=UNITS_A, dim=3, n=(n, n, n), dxi=(d, d, d), bc=("symmetry_lo",) * 3,
                period=(1.0, 1.0, 1.0), x=np.stack([X, Yc, Z]),
                rho=np.where(inside, 1.818, 0.275), v=np.zeros((3,) + X.shape),
                p=np.where(inside, 3.0, 0.575), t_end=t_end, cfl=cfl, moving=moving,
                mesh=dict(monitor="vdw", alphas=(1200.0, 1200.0, 0.0), kappa=2, filter_passes=5,
                          sweeps=10, eps=0.0))


def quadrant_states(seed):
    """Four seeded admissible states near the critical point:
    rho in [0.4, 1.6], p in [0.6, 1.4], |v| <= 0.5 (uniform in the disc), rejection-sampled
    for the recipe acceptance region (supercritical, T >= 1.02) and for every pair of
    neighbouring quadrants."""
    rng = np.random.default_rng(seed)
    while True:
        st = []
        while len(st) < 4:
            rho = rng.uniform(0.4, 1.6)
            p = rng.uniform(0.6, 1.4)
            r = 0.5 * np.sqrt(rng.uniform())
            th = rng.uniform(0.0, 2.0 * np.pi)
            if _recipe_ok(rho, p):
                st.append((rho, r * np.cos(th), r * np.sin(th), p))
        # quadrants: 0 = (x>.5,y>.5), 1 = (x<.5,y>.5), 2 = (x<.5,y<.5), 3 = (x>.5,y<.5)
        if all(_pair_ok(st[i], st[(i + 1) % 4]) for i in range(4)):
            return st


def riemann_2d(n=200, seed=0, t_end=0.2, cfl=0.4, moving=True):
    """2D four-quadrant vdW Riemann problem on [0,1]^2 with outflow boundaries and an
    adaptive moving mesh (monitor with rho and G, alpha = (1200, 1200, 1200), 5 filter
    passes, 5 Jacobi sweeps)."""
    x1, d = uniform_nodes(n, 0.0, 1.0, False)
    X, Yc = np.meshgrid(x1, x1)
    st = quadrant_states(seed)
    q = np.where(X > 0.5, np.where(Yc > 0.5, 0, 3), np.where(Yc > 0.5, 1, 2))
    tab = np.array(st)                    # (4, 4): rho, vx, vy, p
    rho = tab[q, 0]
    v = np.stack([tab[q, 1], tab[q, 2]])
    p = tab[q, 3]
    return dict(gas=UNITS_A, dim=2, n=(n, n), dxi=(d, d), bc=("outflow", "outflow"),
                period=(1.0, 1.0), x=np.stack([X, Yc]), rho=rho, v=v, p=p,
                t_end=t_end, cfl=cfl, moving=moving,
                mesh=dict(monitor="vdw", alphas=(1200.0, 1200.0, 1200.0), kappa=2,
                          filter_passes=5, sweeps=5, eps=0.0))


def riemann_1d(name="RP1", n=100, moving=True, t_end=None, cfl=0.4):
    """1D Riemann problem of Table 5.1 on [0, 1], interface at 0.5, outflow boundaries
    (Example 5.2).  The default final time is the paper's (EXAMPLE_5_2_T_END); the monitor
    weights are the example's (alpha = (1200, 3000, 5000) for RP1 and RP2, 1200 each for RP3,
    kappa = 2 with rho and G); 5 filter passes and 10 sweeps (the example gives neither)."""
    rl, vl, pl, rr, vr, pr = TABLE_5_1[name]
    x, d = uniform_nodes(n, 0.0, 1.0, False)
    left = x < 0.5
    alphas = (1200.0, 3000.0, 5000.0) if name in ("RP1", "RP2") else (1200.0, 1200.0, 1200.0)
    return dict(gas=UNITS_A, dim=1, n=(n,), dxi=(d,), bc=("outflow",), period=(1.0,),
                x=x[None].copy(), rho=np.where(left, rl, rr), v=np.where(left, vl, vr)[None],
                p=np.where(left, pl, pr), t_end=EXAMPLE_5_2_T_END[name] if t_end is None else t_end,
                cfl=cfl, moving=moving,
                mesh=dict(monitor="vdw", alphas=alphas, kappa=2, filter_passes=5,
                          sweeps=10, eps=0.0))


def mach_reflection(case="P1", n1=200, n2=100, variant="MM", t_end=None, cfl=0.4, foot=None):
    """Example 5.4's Mach reflection on [0,1] x [0,0.5] as one reading of an underspecified setup: a planar
    shock whose normal n = (cos theta, -sin theta) points right and down towards the wall y = 0.  Behind
    it, (x - x_f) cos theta - y sin theta < 0, is Table 5.2's left state moving along n with the table's
    v_1 as its normal velocity (times sqrt(8/3): the paper's reduced units to the general ones); ahead is
    the right state at rest.  Wall at y = 0 (a mirrored end), outflow elsewhere.  variant: "MM" (monitor
    with rho and the Laplacian of G, kappa = 1, alpha = (1200, 500)), "MM1" (alpha_2 = 0) or "UM" (fixed
    mesh).  Default foot x_f and final time: D1 0.4 and the paper's t = 0.06 (0.0367 in general units);
    P1 0.1 and 0.04, before the foot leaves the domain."""
    gam, rl, vl, _, pl, rr, vr, _, pr = TABLE_5_2[case]
    th = np.radians(MACH_THETA[case])
    gas = dict(UNITS_A, cv=UNITS_A["R"] / (gam - 1.0))
    x1, d1 = uniform_nodes(n1, 0.0, 1.0, False)
    x2, d2 = uniform_nodes(n2, 0.0, 0.5, False)
    X, Y = np.meshgrid(x1, x2)
    xf = (0.1 if case == "P1" else 0.4) if foot is None else foot
    behind = (X - xf) * np.cos(th) - Y * np.sin(th) < 0.0
    vn = np.sqrt(8.0 / 3.0) * np.where(behind, vl, vr)
    w = dict(gas=gas, dim=2, n=(n2, n1), dxi=(d1, d2), bc=("outflow", "symmetry_lo"), period=(1.0, 0.5),
             x=np.stack([X, Y]), rho=np.where(behind, rl, rr), v=np.stack([vn * np.cos(th), -vn * np.sin(th)]),
             p=np.where(behind, pl, pr), cfl=cfl, moving=variant != "UM",
             t_end=t_end if t_end is not None else (0.04 if case == "P1" else 0.06 * np.sqrt(3.0 / 8.0)))
    if variant != "UM":
        w["mesh"] = dict(monitor="vdw", alphas=(1200.0, 500.0 if variant == "MM" else 0.0), kappa=1,
                         filter_passes=5, sweeps=10, eps=0.0)
    return w


def mm1(w):
    """The MM1 counterpart of a moving-mesh workload (Sec. 5: the monitor without the fundamental
    derivative, alpha_2 = alpha_3 = 0 in eq. van der Waalsmonitor)."""
    m = dict(w["mesh"])
    m["alphas"] = (m["alphas"][0], 0.0, 0.0)
    return dict(w, mesh=m)


def vortex_density(X, Y, t=0.0, eps_v=5.0, period=VORTEX_BOX, center=0.5 * VORTEX_BOX):
    """Density of the isentropic vortex (gamma = 1.4) carried by the mean flow (1, 1) to time t:
    the initial field at (x - t, y - t), wrapped into the periodic box."""
    gam = 1.4
    xb = (X - t - center + 0.5 * period) % period - 0.5 * period
    yb = (Y - t - center + 0.5 * period) % period - 0.5 * period
    r2 = xb * xb + yb * yb
    T = 1.0 - (gam - 1.0) * eps_v ** 2 * np.exp(1.0 - r2) / (8.0 * gam * np.pi ** 2)
    return T ** (1.0 / (gam - 1.0))


def isentropic_vortex(n=64, t_end=1.0, cfl=0.4, eps_v=5.0, box=VORTEX_BOX):
    """Ideal-gas (gamma = 1.4) isentropic vortex centred in the periodic box [0, box)^2, mean flow (1, 1)
    (Shu 1998): dT = -(gamma-1) eps^2 e^(1-r^2) / (8 gamma pi^2),
    dv = eps/(2 pi) e^((1-r^2)/2) (-ybar, xbar), rho = T^(1/(gamma-1)), p = rho T.  The closed form is an
    isolated vortex: in the usual box of side 10 its velocity perturbation is still e^-12 of its peak at the
    edges, and that seam between periodic copies converges at first order, below the scheme's error only
    down to about 1e-8; the default box of side 20 leaves e^-49.5 there."""
    gam = 1.4
    c = 0.5 * box
    x1, d = uniform_nodes(n, 0.0, box, True)
    X, Yc = np.meshgrid(x1, x1)
    xb = X - c
    yb = Yc - c
    r2 = xb**2 + yb**2
    T = 1.0 - (gam - 1.0) * eps_v**2 * np.exp(1.0 - r2) / (8.0 * gam * np.pi**2)
    rho = T ** (1.0 / (gam - 1.0))
    fac = eps_v / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    v = np.stack([1.0 - fac * yb, 1.0 + fac * xb])
    return dict(gas=IDEAL_14, dim=2, n=(n, n), dxi=(d, d), bc=("periodic", "periodic"),
                period=(box, box), x=np.stack([X, Yc]), rho=rho, v=v, p=rho * T,
                t_end=t_end, cfl=cfl, moving=False)


def shock_tube_batch(nprob=4096, lmin=200, lmax=8000, seed=12345, lengths=None, t_ratio_max=1.5):
    """Batched 1D shock tubes on [0, 1], interface at 0.5, outflow boundaries.
    Lengths ~ U{lmin..lmax} (or given); left/right states rho in [0.2, 2.5], p in [0.3, 2],
    v in [-1, 1], rejection-sampled for the recipe acceptance region, between the two states,
    and for a temperature ratio <= t_ratio_max across the interface.  Near the critical point
    a larger temperature jump is a large entropy jump (c_v ln(T_l/T_r) with c_v = 213), and the
    method itself cannot advance such tubes: the interface node leaves the admissible region
    within a few steps in the oracle (39 of 800 unrestricted draws of 200 nodes within ten steps,
    the smallest failing ratio 1.56, none of the 648 draws with the ratio <= 1.5, whatever their
    density ratio)."""
    rng = np.random.default_rng(seed)
    if lengths is None:
        lengths = rng.integers(lmin, lmax + 1, size=nprob)
    lengths = np.asarray(lengths)
    nprob = lengths.size
    states = np.empty((nprob, 6))
    for i in range(nprob):
        while True:
            rl, rr = rng.uniform(0.2, 2.5, 2)
            pl, pr = rng.uniform(0.3, 2.0, 2)
            vl, vr = rng.uniform(-1.0, 1.0, 2)
            Tl, Tr = _recipe_temperature(rl, pl), _recipe_temperature(rr, pr)
            if (_recipe_ok(rl, pl) and _recipe_ok(rr, pr) and _pair_ok((rl, pl), (rr, pr))
                    and max(Tl, Tr) <= t_ratio_max * min(Tl, Tr)):
                break
        states[i] = (rl, vl, pl, rr, vr, pr)
    return dict(gas=UNITS_A, lengths=lengths, states=states)


def batch_fields(batch):
    """Packed initial fields (rho, v, p) of a shock-tube batch: node i of problem k sits at
    off_k + i with x_i = i/(L_k - 1); the left state holds for x < 0.5."""
    L = batch["lengths"]
    rho, v, p = [], [], []
    for k in range(L.size):
        x = np.arange(L[k]) / (L[k] - 1)
        left = x < 0.5
        rl, vl, pl, rr, vr, pr = batch["states"][k]
        rho.append(np.where(left, rl, rr))
        v.append(np.where(left, vl, vr))
        p.append(np.where(left, pl, pr))
    return np.concatenate(rho), np.concatenate(v), np.concatenate(p)


def batch_problem(batch, k, mesh_sweeps=5):
    """Problem k of a batch as a 1D workload (for a per-problem check)."""
    L = int(batch["lengths"][k])
    x, d = uniform_nodes(L, 0.0, 1.0, False)
    rl, vl, pl, rr, vr, pr = batch["states"][k]
    left = x < 0.5
    return dict(gas=batch["gas"], dim=1, n=(L,), dxi=(d,), bc=("outflow",), period=(1.0,), x=x[None].copy(),
                rho=np.where(left, rl, rr), v=np.where(left, vl, vr)[None], p=np.where(left, pl, pr),
                t_end=1e30, cfl=0.4, moving=True,
                mesh=dict(monitor="vdw", alphas=(1200.0, 1200.0, 1200.0), kappa=2, filter_passes=5,
                          sweeps=mesh_sweeps, eps=0.0))


def wavy_mesh_2d(X, Y, amp=0.01):
    """Smooth periodic perturbation of a uniform unit-square mesh (x(X+1, Y) = x + 1)."""
    return np.stack([X + amp * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y),
                     Y + amp * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)])


def mesh_velocity_2d(X, Y, amp=0.05, fixed_edges=False):
    """Smooth mesh-velocity field; zero on the boundary nodes when fixed_edges."""
    xd = amp * np.stack([np.sin(2 * np.pi * (X + Y)), np.cos(2 * np.pi * (X - Y))])
    if fixed_edges:
        xd[:, [0, -1], :] = 0.0
        xd[:, :, [0, -1]] = 0.0
    return xd


def smooth_state_2d(X, Y):
    """Smooth periodic primitive fields (rho, v, p) for operator checks."""
    rho = 0.6 + 0.2 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    v = np.stack([0.3 + 0.1 * np.cos(2 * np.pi * Y), -0.2 + 0.1 * np.sin(2 * np.pi * X)])
    p = 1.0 + 0.1 * np.sin(2 * np.pi * Y)
    return rho, v, p


def rough_state(shape, seed, dim):
    """Seeded random admissible-looking primitive fields (rho, v, p) for stress checks."""
    rng = np.random.default_rng(seed)
    rho = 0.3 + 0.4 * rng.uniform(size=shape)
    v = rng.uniform(-0.5, 0.5, (dim,) + shape)
    p = 0.9 + 0.4 * rng.uniform(size=shape)
    return rho, v, p
