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


def mesh_bytes_per_node(precision, filter_passes, sweeps):
    """Compulsory DRAM bytes per node of one 2D mesh redistribution through es_mesh_redistribute: each kernel of
    the sequence reads its inputs once and writes its outputs once (neighbour reads served from cache).

    FP64 form, in 8-byte words: monitor fields (JU, J -> rho, G) 7, monitor terms (rho, G -> three terms) 5,
    omega 4, each filter pass 2, each Jacobi sweep (omega, x -> x) 5, the limiter inside the last sweep (x^n) 2,
    velocity (x^n, x^mu -> xdot) 6.
    Mixed form, in bytes: the FP32 displacement from x (16 + 8), the fused monitor on the (hi, lo) state
    (40 + 12), omega and all filter passes in one tile kernel (12 + 4), all Jacobi sweeps and the limiter in
    one tile kernel (omega, d -> d: 4 + 8 + 8; the limiter reads the sweeps' own values), velocity (d, d^mu ->
    float and double xdot: 16 + 8 + 16)."""
    if precision == "fp64":
        return 8 * (7 + 5 + 4 + 2 * filter_passes + 5 * sweeps + 2 + 6)
    return 24 + 52 + 16 + 20 + 40
