// es_stage_mixed.cu -- the fused operator + SSP-RK3 stage in the mixed-precision form.
//
// GB300 runs FP32 about 70 times faster than FP64 (2 FP64 FMA lanes per SM per
// clock), and an FP64 -> FP32 conversion costs as much as an FP64 FMA.  This
// form therefore keeps the per-stage work entirely on the FP32 pipe:
//   * the state JU, J is stored as compensated pairs of floats (hi, lo), value
//     hi + lo with a 48-bit significand, in two planes [2][...] (hi plane first);
//     the primitive state (rho, v, T) and the RK combination are evaluated in
//     double-float arithmetic (error-free sums and products built from FP32
//     FMA), so the jumps of rho, v and T between neighbouring nodes keep their
//     digits even where they are far below the FP32 resolution of the values
//     (near smooth extrema); everything else is plain FP32 on the hi parts;
//   * the mesh enters as an FP32 displacement d = x - (x_00 + i dxi_1, y_00 + j dxi_2)
//     and an FP32 mesh velocity, converted from the FP64 mesh once per step, so
//     the metric differences delta_k[x] = dxi_k e_k + delta_k[d] lose no digits;
//   * logarithmic means are taken per pair from the relative jump
//     f = (a_l - a_r)/(a_l + a_r) (series for |f| < 0.05, log1p otherwise), which
//     is accurate to FP32 rounding of the result even for nearly equal states;
//   * the entropy variables never appear as absolute values (V_1 is O(c_v) =
//     O(200) and its jumps are O(h)): the dissipation works on the jumps
//     V_j - V_i written exactly as the jump decomposition of Sec. 3.1
//     (eq. jumpV, general units), and MR-WENO5 is applied to W_j - W_i, which
//     it reconstructs exactly as it would W_j (the reconstruction commutes with
//     adding a constant).
// What stays FP64 is the once-per-step mesh conversion and the mesh
// redistribution kernels.
#include <cuda_runtime.h>

#include "es_mixed_device.cuh"

namespace es {

namespace {

using namespace mixed;

// resident CTAs per SM the register allocation must allow: 5 x 160 or 4 x 192 threads (24 warps; 72 and 80
// registers, no spills), 2 x 320 or 384 (the two-lanes-per-face shapes), 1 x 544
template <int DIM, int BX, int BY, int NT, bool SPLIT>
__global__ void __launch_bounds__(NT, NT <= 160 ? 5 : (NT <= 192 ? 4 : (NT <= 384 ? 2 : 1)))
    stage_kernel_mixed(StageParams P) {
    extern __shared__ float smemf[];
    const int ntx = (P.n1 + BX - 1) / BX;
    const int i0 = (blockIdx.x % ntx) * BX;
    const int j0 = DIM == 2 ? (blockIdx.x / ntx) * BY : 0;
    const double dtd = P.dt_dev ? *P.dt_dev : P.dt_host;
    if (P.mode == 0 && dtd == 0.0) return;               // finished run: leave the state untouched
    stage_tile_mixed<DIM, BX, BY, NT, SPLIT>(smemf, P, i0, j0, float(dtd), gas_f(P), weno_f(P));
}

template <int DIM, int BX, int BY, int NT, bool SPLIT = false>
cudaError_t prepare_tile_f() {
    return cudaFuncSetAttribute(stage_kernel_mixed<DIM, BX, BY, NT, SPLIT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(TileF<DIM, BX, BY, NT>::SMEM));
}

template <int DIM, int BX, int BY, int NT, bool SPLIT = false>
cudaError_t launch_tile_f(const StageParams& P, cudaStream_t s) {
    const int ntx = (P.n1 + BX - 1) / BX;
    const int nty = DIM == 2 ? (P.n2 + BY - 1) / BY : 1;
    stage_kernel_mixed<DIM, BX, BY, NT, SPLIT><<<ntx * nty, NT, TileF<DIM, BX, BY, NT>::SMEM, s>>>(P);
    return cudaGetLastError();
}

}  // namespace

// 2D shapes: 20 x 8 nodes with 384 threads, two lanes per face (twice the warps of the 192-thread
// shape: small meshes are latency bound), 25 x 6 with 192 (175 faces; 8 x 34 = 272 tiles fill
// 200 x 200 at two CTAs per SM in one wave), 20 x 8 with 192 (180 faces), 20 x 14 with 608, two lanes
// per face (10 x 15 = 150 tiles: one CTA on each SM at 200 x 200, less halo per node), and 16 x 8 with 160
// (more CTAs for small meshes)
cudaError_t stage_prepare_mixed(int dim) {
    if (dim == 1) return prepare_tile_f<1, 254, 1, 256>();
    cudaError_t e = prepare_tile_f<2, 20, 8, 384, true>();
    if (e == cudaSuccess) e = prepare_tile_f<2, 25, 6, 192>();
    if (e == cudaSuccess) e = prepare_tile_f<2, 20, 8, 192>();
    if (e == cudaSuccess) e = prepare_tile_f<2, 20, 14, 608, true>();
    if (e == cudaSuccess) e = prepare_tile_f<2, 16, 8, 160>();
    return e;
}

cudaError_t launch_stage_mixed(const StageParams& P, cudaStream_t s) {
    if (P.dim == 1) return launch_tile_f<1, 254, 1, 256>(P, s);
    switch (P.tile) {
        case 1: return launch_tile_f<2, 25, 6, 192>(P, s);
        case 2: return launch_tile_f<2, 20, 8, 192>(P, s);
        case 3: return launch_tile_f<2, 20, 14, 608, true>(P, s);
        case 4: return launch_tile_f<2, 16, 8, 160>(P, s);
        default: return launch_tile_f<2, 20, 8, 384, true>(P, s);
    }
}

}  // namespace es
