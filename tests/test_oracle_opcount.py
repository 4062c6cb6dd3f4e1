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
