"""The FP64 entropy production check (es_entropy_rate) against the oracle's total entropy rate.

For (dJU, dJ) the right-hand sides of eq. semi_U / semi_J, d/dt sum_i J_i eta(U_i) dV = dV sum_i (V_i . dJU_i -
phi_i dJ_i).  On periodic data the EC scheme conserves it (eq. ECCondition_comp: the EC fluxes telescope), so it is
round-off of the magnitude of its terms; the ES flux (eq. HOstable) makes it negative.  The library's value equals
the oracle's to 1e-12 of that magnitude, on fixed and moving meshes, in one, two and three dimensions.
"""
import numpy as np
import pytest

from oracle import operator as op
from paper_2407_05568_gb300 import workloads as wl

from sides import gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_05568_gb300 import build
    build.build()


def _case(name):
    if name == "sine1d_rough":
        w = wl.sine_1d(64)
        w["rho"], w["v"], w["p"] = wl.rough_state((64,), 5, 1)
        w["xdot"] = np.zeros_like(w["x"])
    elif name == "wavy2d_moving":
        w = wl.sine_2d(40)
        X, Y = w["x"]
        w["x"] = wl.wavy_mesh_2d(X, Y)
        w["rho"], w["v"], w["p"] = wl.rough_state(X.shape, 9, 2)
        w["xdot"] = wl.mesh_velocity_2d(X, Y)
    else:                                     # 3D periodic, rough state, moving mesh
        w = wl.sine_3d(10)
        X, Y, Z = w["x"]
        w["rho"], w["v"], w["p"] = wl.rough_state(X.shape, 13, 3)
        tp = 2 * np.pi
        w["xdot"] = 0.05 * np.stack([np.sin(tp * (X + Y)), np.cos(tp * (Y - Z)), np.sin(tp * (Z + X))])
    return w


def _rates(w, dissipation, precision="fp64"):
    import torch

    from paper_2407_05568_gb300 import es
    sch, mc, JU_o, J_o, x = oracle_setup(w, dissipation=dissipation)
    dU_o, dJ_o = op.rhs(sch, JU_o, J_o, x, w["xdot"])
    rate_o = op.entropy_rate(sch, JU_o, J_o, dU_o, dJ_o)
    ctx, JU, J, xt = gpu_setup(w, precision=precision, dissipation=dissipation)
    xd = torch.tensor(np.ascontiguousarray(w["xdot"]), dtype=torch.float64, device="cuda")
    dU, dJ = torch.empty_like(JU), torch.empty_like(J)
    es.es_rhs(ctx, JU, J, xt, xd, dU, dJ)
    rate_g, scale_g = es.es_entropy_rate(ctx, JU, J, dU, dJ)
    again = es.es_entropy_rate(ctx, JU, J, dU, dJ)
    assert again == (rate_g, scale_g)                     # fixed-order reduction: the same bits
    assert es.es_check(ctx) == 0
    return rate_o, rate_g, scale_g


@pytest.mark.parametrize("case", ["sine1d_rough", "wavy2d_moving", "rough3d_moving"])
def test_ec_scheme_conserves_entropy(case):
    rate_o, rate_g, scale = _rates(_case(case), dissipation=False)
    assert scale > 0.0
    assert abs(rate_g) <= 1e-12 * scale, (rate_g, scale)
    assert abs(rate_g - rate_o) <= 1e-12 * scale


@pytest.mark.parametrize("case", ["sine1d_rough", "wavy2d_moving", "rough3d_moving"])
def test_es_scheme_produces_entropy(case):
    rate_o, rate_g, scale = _rates(_case(case), dissipation=True)
    assert rate_g < -1e-6 * scale, (rate_g, scale)
    assert abs(rate_g - rate_o) <= 1e-12 * scale, (rate_g, rate_o, scale)


def test_mixed_form_rate_in_fp64():
    """The mixed form's right-hand sides carry FP32 flux rounding (~1e-6 of the flux scale); the check itself reads
    the (hi, lo) planes in FP64, so its value is the oracle's within that rounding and keeps the sign."""
    rate_o, rate_g, scale = _rates(_case("wavy2d_moving"), dissipation=True, precision="mixed")
    assert rate_g < 0.0
    assert abs(rate_g - rate_o) <= 1e-5 * scale, (rate_g, rate_o, scale)
