"""Example 5.4's Mach reflection (a reading of its geometry; see the workload): full FP64 steps with the
wall at y = 0 through es_steps against the oracle, in the MM, MM1 and UM variants."""
import numpy as np
import pytest

from oracle import stepper
from paper_2407_05568_gb300 import workloads as wl
from sides import gpu_setup, oracle_setup, rel_l1, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["P1", "D1"])
@pytest.mark.parametrize("variant", ["MM", "MM1", "UM"])
def test_mach_reflection_steps_against_oracle(case, variant):
    from paper_2407_05568_gb300 import es
    w = wl.mach_reflection(case, 61, 33, variant)
    sch, mc, JU_o, J_o, x_o = oracle_setup(w)
    ctx, JU, J, xt = gpu_setup(w)
    nsteps = 3
    t = 0.0
    for _ in range(nsteps):
        JU_o, J_o, x_o, t, _ = stepper.step(sch, mc, JU_o, J_o, x_o, t, w["t_end"], w["cfl"])
    es.es_set_time(ctx, 0.0)
    es.es_steps(ctx, JU, J, xt, nsteps, w["t_end"])
    assert es.es_check(ctx) == 0, es.es_last_error(ctx)
    tg, _ = es.es_get_time(ctx)
    assert abs(tg - t) <= 1e-12 * t
    assert rel_l1(to_np(JU), JU_o) < 1e-12 * nsteps
    assert np.abs(to_np(xt) - x_o).max() < 1e-12
    if variant != "UM":
        assert np.abs(x_o - w["x"]).max() > 1e-3 * w["dxi"][0]      # the mesh moved


def test_mach_reflection_mixed_form_is_rejected():
    """The wall is a mirrored end, which the mixed form does not have."""
    from paper_2407_05568_gb300 import es
    with pytest.raises(es.EsError):
        gpu_setup(wl.mach_reflection("P1", 61, 33, "MM"), precision="mixed")
