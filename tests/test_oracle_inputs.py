"""What the batched input recipe excludes, and why: the method itself (the oracle) cannot advance those inputs.

The batched shock tubes draw rho in [0.2, 2.5], p in [0.3, 2], v in [-1, 1], keep supercritical states, and keep a
temperature ratio <= 1.5 across the interface.  Near the critical point a larger temperature jump is a large entropy
jump (c_v = R/0.0125 = 213), and the high-order ES scheme (eq. HOstable) then drives the interface node out of the
admissible region (eq. coefflimit) within a few steps.  The failure does not depend on the points where the paper is
silent about the dissipation (the sign switch's dead zone, the assignment of the MR-WENO linear weights).  Density
ratios need no cap.
"""
import numpy as np
import pytest

from oracle import operator as op
from oracle import stepper, thermo
from paper_2407_05568_gb300 import workloads as wl

from sides import oracle_setup


def _stays_admissible(w, steps, **scheme):
    sch, mc, JU, J, x = oracle_setup(w)
    if scheme:
        sch = op.Scheme(**{**sch.__dict__, **scheme})
    t = 0.0
    for _ in range(steps):
        with np.errstate(invalid="ignore", divide="ignore"):
            JU, J, x, t, _ = stepper.step(sch, mc, JU, J, x, t, 1e30, w["cfl"])
            rho, v, T, p = thermo.cons_to_prim(sch.gas, JU / J)
            ok = thermo.admissible(sch.gas, rho, T) & np.isfinite(rho) & np.isfinite(T)
        if not ok.all():
            return False
    return True


def _uncapped(n=800, length=200):
    return wl.shock_tube_batch(nprob=n, lengths=np.full(n, length), seed=777, t_ratio_max=1e9)


def _t_ratio(st):
    Tl = wl._recipe_temperature(st[0], st[2])
    Tr = wl._recipe_temperature(st[3], st[5])
    return max(Tl, Tr) / min(Tl, Tr)


@pytest.mark.parametrize("k", [292, 255])
def test_draws_above_the_temperature_cap_fail_in_the_oracle(k):
    """Draws 292 and 255 of an uncapped batch (temperature ratios 1.56 and 1.70, the two smallest among the failing
    draws of 800) leave the admissible region within ten oracle steps."""
    b = _uncapped()
    assert 1.5 < _t_ratio(b["states"][k]) < 1.75
    assert not _stays_admissible(wl.batch_problem(b, k), 10)


def test_failure_does_not_depend_on_the_dissipation_readings():
    """Draw 292 fails as well without the sign switch's dead zone (sign_tol = 0) and with the MR-WENO linear weights
    equal or in the reverse order."""
    w = wl.batch_problem(_uncapped(), 292)
    assert not _stays_admissible(w, 10, sign_tol=0.0)
    assert not _stays_admissible(w, 10, weno_gammas=(1 / 3, 1 / 3, 1 / 3))
    assert not _stays_admissible(w, 10, weno_gammas=(0.95, 0.045, 0.005))


def test_capped_recipe_runs_whatever_the_density_ratio():
    """With the recipe's temperature cap, the six draws with the largest density ratios among 400 (ratios above 5)
    and six ordinary draws stay admissible over ten steps."""
    b = wl.shock_tube_batch(nprob=400, lengths=np.full(400, 200), seed=4)
    st = b["states"]
    ratio = np.maximum(st[:, 0], st[:, 3]) / np.minimum(st[:, 0], st[:, 3])
    picks = list(np.argsort(ratio)[-6:]) + list(range(6))
    assert ratio[picks[0]] > 5.0
    for k in picks:
        assert _t_ratio(st[k]) <= 1.5
        assert _stays_admissible(wl.batch_problem(b, int(k)), 10), k
