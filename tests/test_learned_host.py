"""Host logic of the learned warm start's evaluation (no GPU): the matched-accuracy interpolation."""
import numpy as np

from paper_2407_05568_gb300 import learned


def _res(points):
    """compare_matched's per-tolerance records from (tolerance, mean distance, mean sweeps) triples."""
    return {t: {"dist_plain_mean": np.array([d, d]), "sweeps_plain": np.array([s, s])} for t, d, s in points}


def test_plain_at_interpolates_log_log_between_tolerances():
    # sweeps ~ dist^-1/2 and tol ~ dist: log-log interpolation is exact for power laws
    pts = [(t, 10.0 * t, 3.0 / np.sqrt(10.0 * t)) for t in (0.02, 0.01, 0.005, 0.0025)]
    res = _res(pts)
    tol, sw = learned.plain_at(res, 0.07)
    assert np.isclose(tol, 0.007, rtol=1e-12)
    assert np.isclose(sw, 3.0 / np.sqrt(0.07), rtol=1e-12)
    # at a sampled distance it returns the sample
    tol, sw = learned.plain_at(res, 0.05)
    assert np.isclose(tol, 0.005) and np.isclose(sw, 3.0 / np.sqrt(0.05))


def test_plain_at_outside_the_sampled_range_is_none():
    res = _res([(0.02, 0.2, 4.0), (0.01, 0.1, 6.0)])
    assert learned.plain_at(res, 0.3) is None
    assert learned.plain_at(res, 0.05) is None
    assert learned.plain_at(res, 0.2) == (0.02, 4.0)
