"""The roofline's operation counts per node and RK stage are the oracle's (oracle/opcount.py), recomputed here."""
import pytest

from oracle import opcount
from paper_2407_05568_gb300 import perfmodel


@pytest.mark.parametrize("dim", [1, 2])
def test_stage_operation_count_is_the_oracles(dim):
    total, pair = opcount.per_node_stage(dim)
    assert perfmodel.COUNTS[dim]["total"] == pytest.approx(total, rel=5e-3)
    assert perfmodel.COUNTS[dim]["pair"] == pytest.approx(pair, rel=5e-3)
    assert perfmodel.flops_per_node_stage(dim) == perfmodel.COUNTS[dim]["total"]


def test_counter_counts_a_known_expression():
    """The tallying arrays count one operation per element of +, -, *, /, sqrt, log and two per contraction term."""
    import numpy as np
    a = np.linspace(1.0, 2.0, 10).view(opcount.Counted)
    with opcount._counting() as t:
        b = np.sqrt(a * a + 1.0) / a                    # 4 per element
        c = np.log(b) - np.abs(b)                       # 2 per element (abs counts nothing)
        np.einsum("i,i->", a, c)                        # 10 terms: 20
        np.where(c > 0, c, -c)                          # selection and comparison: 0
    assert t.total == 40 + 20 + 20


def test_mesh_bytes_per_node_counts_each_kernels_inputs_and_outputs():
    """The mesh roofline's compulsory bytes: the FP64 form's kernel sequence in 8-byte words (monitor fields
    JU[4], J -> rho, G; terms rho, G -> 3; omega 3 -> 1; per filter pass 1 -> 1; per sweep omega, x[2] -> x[2];
    the limiter inside the last sweep x^n[2]; velocity x^n[2], x^mu[2] -> xdot[2]) and the mixed form's fused sequence in bytes
    (displacement x[2] double -> d[2] float; monitor on the (hi, lo) state JU[4], J -> 3 float terms; omega with
    its passes 3 -> 1 float; sweeps with the limiter omega, d[2] -> d[2]; velocity d[2], d^mu[2] -> float and
    double xdot[2])."""
    from paper_2407_05568_gb300 import perfmodel
    words = (5 + 2) + (2 + 3) + (3 + 1) + 5 * (1 + 1) + 5 * (1 + 2 + 2) + 2 + (2 + 2 + 2)
    assert perfmodel.mesh_bytes_per_node("fp64", 5, 5) == 8 * words
    mixed = (16 + 8) + (5 * 8 + 12) + (12 + 4) + (4 + 8 + 8) + (16 + 8 + 16)
    assert perfmodel.mesh_bytes_per_node("mixed", 5, 5) == mixed
    # one more pass or sweep adds its traffic in the FP64 form; the fused mixed kernels read and write once
    assert perfmodel.mesh_bytes_per_node("fp64", 6, 5) - perfmodel.mesh_bytes_per_node("fp64", 5, 5) == 16
    assert perfmodel.mesh_bytes_per_node("fp64", 5, 6) - perfmodel.mesh_bytes_per_node("fp64", 5, 5) == 40
    assert perfmodel.mesh_bytes_per_node("mixed", 8, 8) == mixed
