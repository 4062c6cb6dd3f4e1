"""Example 5.2: the 1D van der Waals Riemann problems of Table 5.1, run by the oracle to the paper's final times.

The paper states what each solution shows at its final time (Sec. 5, Example 5.2); those statements are the pins:
  * RP1 (t = 0.15 Z_c^(-1/2)): G > 0 at first; G < 0 emerges (a transonic rarefaction fan and a rarefaction
    shock), and G changes sign near x_1 = 0.74, where a compressive shock forms;
  * RP2 (t = 0.45 Z_c^(-1/2)): G stays negative in the whole flow field during the whole evolution;
  * RP3 (t = 0.2 Z_c^(-1/2)): a G < 0 region and a G > 0 region.
The example runs them as MM and MM1 with 100 cells and as UM with 300; so do these tests.  Beyond the paper's
statements:
  * every node stays admissible (eq. coefflimit) after every step;
  * on the fixed mesh, eq. semi_U in conservation form fixes the totals.  Mass and energy are conserved.  The
    momentum grows by the pressure force of the two unperturbed end states, (p_l - p_r) t, with Table 5.1's
    pressures.  Waves reach neither end by the final time;
  * on the moving mesh, J (advanced only by the VCL, eq. semi_J) still equals the Jacobian delta_1[x] of the
    final mesh after the whole run.
Final times: the paper's are in its reduced units, whose velocities are sqrt(3/8) of the ones used here, so
0.15 Z_c^(-1/2) with Z_c = 3/8 is t = 0.15 here (likewise 0.45 and 0.2).
"""
import functools

import numpy as np
import pytest

from oracle import operator as op
from oracle import stepper, thermo
from paper_2407_05568_gb300 import workloads as wl

from sides import oracle_setup

VARIANTS = {"MM": 100, "MM1": 100, "UM": 300}


def _workload(name, variant):
    w = wl.riemann_1d(name, n=VARIANTS[variant], moving=variant != "UM")
    return wl.mm1(w) if variant == "MM1" else w


@functools.lru_cache(maxsize=None)
def _run(name, variant):
    """The oracle run to the final time; per step the extreme G and whether every node is admissible."""
    w = _workload(name, variant)
    sch, mc, JU, J, x = oracle_setup(w)
    g = sch.gas
    t = 0.0
    steps = 0
    g_max, admissible = -np.inf, True
    while t < w["t_end"] * (1.0 - 1e-14):
        JU, J, x, t, _ = stepper.step(sch, mc, JU, J, x, t, w["t_end"], w["cfl"])
        steps += 1
        rho, v, T, p = thermo.cons_to_prim(g, JU / J)
        admissible &= bool(np.all(thermo.admissible(g, rho, T)))
        g_max = max(g_max, float(np.max(thermo.fundamental_derivative(g, rho, T))))
    rho, v, T, p = thermo.cons_to_prim(g, JU / J)
    G = thermo.fundamental_derivative(g, rho, T)
    return dict(w=w, sch=sch, JU=JU, J=J, x=x, t=t, steps=steps, G=G, G_max_run=g_max, admissible=admissible)


CASES = [(name, variant) for name in ("RP1", "RP2", "RP3") for variant in VARIANTS]


@pytest.mark.parametrize("name,variant", CASES)
def test_runs_to_final_time_admissible(name, variant):
    r = _run(name, variant)
    assert r["t"] == pytest.approx(wl.EXAMPLE_5_2_T_END[name], rel=1e-13)
    assert r["admissible"]
    assert np.all(np.isfinite(r["JU"]))


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_rp1_sign_change_of_g_near_074(variant):
    """RP1: G > 0 in both initial states (Table 5.1: 4.118, 0.703); at the final time G < 0 between the
    transonic rarefaction and the shock, and G turns positive again at the shock, near x_1 = 0.74."""
    r = _run("RP1", variant)
    G, x = r["G"], r["x"][0]
    assert G[0] > 4.0 and G[-1] > 0.6
    assert G.min() < -0.5
    cross = np.where(np.diff(np.sign(G)) > 0)[0]          # - to + crossings, left to right
    assert cross.size >= 1
    xs = 0.5 * (x[cross[-1]] + x[cross[-1] + 1])
    assert 0.70 < xs < 0.78, xs


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_rp2_g_negative_throughout(variant):
    """RP2: the fundamental derivative keeps negative in the whole flow field during the evolution.  That is a
    statement about the solution; a discretisation overshoots at its discontinuities.  On the moving meshes G stays
    below 5e-3 over the whole run (a few early steps at the initial jump) and is negative everywhere at the final
    time.  On the uniform mesh at most two nodes at the rarefaction shock overshoot, by < 0.1, against a range of
    G from -1.4 to -0.02."""
    r = _run("RP2", variant)
    G = r["G"]
    assert G.min() < -1.0
    if variant == "UM":
        assert np.count_nonzero(G > 0.0) <= 2 and G.max() < 0.1
        assert r["G_max_run"] < 0.1
    else:
        assert G.max() < 0.0
        assert r["G_max_run"] < 5e-3


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_rp3_g_changes_sign(variant):
    """RP3: a G < 0 region (left state G = -0.031) and a G > 0 region (right state G = 0.703) at the final time,
    with a single sign change between them."""
    r = _run("RP3", variant)
    G = r["G"]
    assert G.min() < -0.02 and G.max() > 0.6
    assert G[0] < 0.0 < G[-1]


@pytest.mark.parametrize("name", ["RP1", "RP2", "RP3"])
def test_fixed_mesh_totals(name):
    """UM: the mass and energy totals are conserved; the momentum total equals (p_l - p_r) t_end (the flux through
    each end is F(U) of its unperturbed state, whose only nonzero entry is the pressure)."""
    r = _run(name, "UM")
    w, sch = r["w"], r["sch"]
    J0 = op.node_jacobian(sch, w["x"])
    U0 = thermo.prim_to_cons(sch.gas, w["rho"], w["v"], w["p"]) * J0
    tot0 = U0.sum(axis=1) * sch.dxi[0]
    tot1 = r["JU"].sum(axis=1) * sch.dxi[0]
    assert abs(tot1[0] - tot0[0]) <= 1e-8 * tot0[0]
    assert abs(tot1[2] - tot0[2]) <= 1e-8 * tot0[2]
    rl, vl, pl, rr, vr, pr = wl.TABLE_5_1[name]
    force = (pl - pr) * r["t"]
    assert abs(tot1[1] - force) <= 1e-7 * abs(force)


@pytest.mark.parametrize("name", ["RP1", "RP2", "RP3"])
def test_moving_mesh_j_equals_jacobian_of_the_mesh(name):
    """MM: J, advanced only by the discrete VCL over several hundred steps, equals delta_1[x] of the final mesh;
    the mesh stays ordered and its ends stay at 0 and 1."""
    r = _run(name, "MM")
    sch, x = r["sch"], r["x"]
    Jg = op.node_jacobian(sch, x)
    assert np.abs(r["J"] - Jg).max() <= 1e-11 * np.abs(Jg).max()
    assert np.all(np.diff(x[0]) > 0.0)
    assert x[0, 0] == 0.0 and x[0, -1] == 1.0
    assert r["steps"] > 300
