"""Algorithmic work per node and RK stage of the fused stage kernel, and the peaks it is compared to.

Operation counts are taken from the formulas the kernel evaluates (es_stage.cu),
counting one operation per +, -, *, /, sqrt and log and two per fused
multiply-add.  They count each algorithmic quantity once per node (node data),
three pairs per node and direction (the pair fluxes F(U_i, U_{i+m}), m = 1..3)
and one face per node and direction; the halo recomputation of a tiled kernel
is not algorithmic work and is not counted.

Per node (2D):
  node data      61   primitive state, 1/T, 1/(1 - b rho), four logarithms, entropy variables
  metrics        34   two 6th-order differences per direction and J xi_t
  pair flux     120   x 6 (3 per direction): means, three inverse log means
                      (series branch 17, log branch 4; a typical mix), D, U~_1, F~_1,
                      and the contraction with the face metrics
  face flux    1470   x 2: the alpha-combination of six pairs (72), the face
                      eigen-system (~110), six projections W = R^T T V (192),
                      eight MR-WENO5 reconstructions (129 each = 1032),
                      sign switch and back-projection (~50)
  divergence     55   two directions and the Shu-Osher combination
  total        3810
Per node (1D): node 44, metrics 2, pair 75 x 3, face 1000 x 1, divergence 20 -> 1291.
"""

COUNTS = {
    2: dict(node=61, metrics=34, pair=120, pairs=6, face=1470, faces=2, rk=55),
    1: dict(node=44, metrics=2, pair=75, pairs=3, face=1000, faces=1, rk=20),
}


def flops_per_node_stage(dim):
    c = COUNTS[dim]
    return c["node"] + c["metrics"] + c["pair"] * c["pairs"] + c["face"] * c["faces"] + c["rk"]


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
