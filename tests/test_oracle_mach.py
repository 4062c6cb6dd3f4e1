"""Pins of the Mach-reflection workload (Example 5.4, Table 5.2; its geometry is a reading).

Table 5.2's states are read as the two sides of a planar shock with v_1 the velocity along the shock
normal, in the paper's reduced units (velocities times sqrt(8/3) in the general units).  The
Rankine-Hugoniot conditions then hold in the frame of the shock: with the shock speed s fixed by the
mass flux, the momentum flux rho (v - s)^2 + p and the enthalpy e + p/rho + (v - s)^2/2 agree on the
two sides to the table's rounding (three or four digits)."""
import numpy as np
import pytest

from oracle import thermo
from paper_2407_05568_gb300 import workloads as wl


@pytest.mark.parametrize("case", ["P1", "D1"])
def test_table_5_2_states_are_a_shock_in_its_normal_frame(case):
    gam, rl, vl, v2l, pl, rr, vr, v2r, pr = wl.TABLE_5_2[case]
    assert v2l == 0.0 and v2r == 0.0 and vr == 0.0
    g = thermo.Gas(a=3.0, b=1.0 / 3.0, R=8.0 / 3.0, cv=(8.0 / 3.0) / (gam - 1.0))
    va = vl * np.sqrt(8.0 / 3.0)
    s = rl * va / (rl - rr)                                  # mass flux continuous
    side = []
    for rho, v, p in ((rl, va, pl), (rr, 0.0, pr)):
        U = thermo.prim_to_cons(g, np.array([rho]), np.array([[v]]), np.array([p]))
        e = U[-1, 0] / rho - 0.5 * v * v
        side.append((rho * (v - s) ** 2 + p, e + p / rho + 0.5 * (v - s) ** 2))
    (mom_l, h_l), (mom_r, h_r) = side
    assert abs(mom_l - mom_r) < 5e-3 * mom_r
    assert abs(h_l - h_r) < 5e-3 * abs(h_r)
    # the shock moves into the right state: P1 a compression shock, D1 a rarefaction shock (non-classical,
    # the post-shock side is the lower-density one and moves against the shock)
    assert s > 0.0
    assert (rl > rr) == (case == "P1")


@pytest.mark.parametrize("case", ["P1", "D1"])
def test_mach_reflection_initial_state(case):
    """Behind the front the left state moves along the normal (cos theta, -sin theta); ahead the right
    state is at rest; the wall is the mirrored low end of xi_2."""
    w = wl.mach_reflection(case, 60, 30, "MM")
    th = np.radians(wl.MACH_THETA[case])
    gam, rl, vl, _, pl, rr, _, _, pr = wl.TABLE_5_2[case]
    behind = w["rho"] == rl
    assert behind.any() and (~behind).any() and w["bc"] == ("outflow", "symmetry_lo")
    vn = vl * np.sqrt(8.0 / 3.0)
    assert np.allclose(w["v"][0][behind], vn * np.cos(th)) and np.allclose(w["v"][1][behind], -vn * np.sin(th))
    assert np.all(w["v"][:, ~behind] == 0.0) and np.all(w["p"][behind] == pl) and np.all(w["p"][~behind] == pr)
    X, Y = w["x"]
    assert np.all(((X - 0.1 if case == "P1" else X - 0.4) * np.cos(th) - Y * np.sin(th) < 0) == behind)
    assert wl.mach_reflection(case, 60, 30, "MM1")["mesh"]["alphas"] == (1200.0, 0.0)
    assert not wl.mach_reflection(case, 60, 30, "UM")["moving"]
