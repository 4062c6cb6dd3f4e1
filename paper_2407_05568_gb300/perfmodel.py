"""Algorithmic work per node and RK stage of the fused stage kernel, and the peaks it is compared to.

The counts are the oracle's: oracle/opcount.py runs one RK stage of the oracle on arrays that tally every
elementwise floating-point operation (+, -, *, /, square roots, logarithms and other transcendental functions one
each, an FMA two, selections and comparisons none, contractions one multiply and one add per term), divides the
pair fluxes' operations by their reuse (the oracle evaluates each pair once per face that uses it, the algorithm
once), and takes the per-node coefficient of a fit over three mesh sizes, which removes the ghost nodes' work.
tests/test_oracle_opcount.py recomputes them against the numbers below.

They exceed the count of the kernel's own formulas (1291 in 1D, 3810 in 2D: node data 61, metrics 34, 6 pairs x 120,
2 faces x 1470, divergence and RK 55), which shares node data between the two directions, forms one rotation per
node and evaluates the smoothness indicators from differences; the oracle's plain evaluation is the algorithm's
work, the kernel's count is what it issues (plus halo recomputation).
"""

COUNTS = {
    2: dict(total=4837, pair=1212),
    1: dict(total=1707, pair=480),
}
KERNEL_FORMULA_COUNTS = {2: 3810, 1: 1291}


def flops_per_node_stage(dim):
    return COUNTS[dim]["total"]


def stage_flops(dim, nodes, precision="fp64"):
    """Algorithmic operations of one stage-kernel launch over `nodes` nodes."""
    return flops_per_node_stage(dim) * nodes


GB300_SMS = 152
GB300_MAX_SM_MHZ = 2070.0


def fp64_peak_tflops(peaks=None):
    """Nominal FP64 rate of GB300 (1.25 TFLOP/s, the profiling recipe's figure)."""
    return 1.25


def fp32_peak_tflops(peaks=None):
    """152 SMs x 128 FP32 lanes x 2 (FMA) x the maximum SM clock."""
    mhz = (peaks or {}).get("sm_max_mhz", GB300_MAX_SM_MHZ)
    return GB300_SMS * 128 * 2 * mhz * 1e6 / 1e12
