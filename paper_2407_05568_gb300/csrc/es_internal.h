// es_internal.h -- host/device structures shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "es_device.cuh"
#include "es_vdw.h"

namespace es {

// Arguments of the fused operator / RK-stage kernels.
struct StageParams {
    int dim;
    int n1, n2;
    int bc[2];
    double inv_dxi[2];
    double period[2];
    Gas gas;
    Weno weno;
    int diss;
    double ca, cb, cst;           // a_s, b_s, c_s of SSP-RK3
    double dt_host;
    const double* dt_dev;         // device dt (nullptr: use dt_host)
    const double* JUn;            // read at the node only
    const double* Jn;
    const double* JUs;            // read with the halo
    const double* Js;
    const double* xn;             // mesh at t^n (halo)
    const double* xdot;           // mesh velocity (nullable)
    double* JUo;
    double* Jo;
    int mode;                     // 0: RK combination; 1: write the right-hand sides
    int tile;                     // 2D tile shape: index into the precision's shape table
    DevStatus* status;
    // mixed form: float state and float mesh displacement / velocity
    const float* fJUn;
    const float* fJn;
    const float* fJUs;
    const float* fJs;
    float* fJUo;
    float* fJo;
    const float* fdisp;           // x - (x_00 + i dxi_1, y_00 + j dxi_2), [dim][n2][n1]
    const float* fxdot;           // mesh velocity, [dim][n2][n1] (nullable)
    // float copies of the constants (GB300 converts double -> float at FP64 speed)
    float fgas[9];                // a, b, R, cv, delta, R b, 1/cv, 1/R, 1/delta
    float fweno[8];               // g1, g2, g3, g12, ig22, ig3, eps, sign_tol
    float finv_dxi[2];
    float fca, fcb, fca_lo, fcb_lo, fcst;
    // mixed form strides: component stride, JU lo-plane offset, J lo-plane offset
    // (0: the contiguous layout of one mesh, n1 n2, (dim + 2) n1 n2 and n1 n2)
    size_t fcs, fps, fpsJ;
};

// fill the float copies of the constants of a stage launch
inline void set_float_params(StageParams& P) {
    P.fgas[0] = float(P.gas.a);
    P.fgas[1] = float(P.gas.b);
    P.fgas[2] = float(P.gas.R);
    P.fgas[3] = float(P.gas.cv);
    P.fgas[4] = float(P.gas.delta);
    P.fgas[5] = float(P.gas.R * P.gas.b);
    P.fgas[6] = float(1.0 / P.gas.cv);
    P.fgas[7] = float(1.0 / P.gas.R);
    P.fgas[8] = float(P.gas.cv / P.gas.R);
    const double w[8] = {P.weno.g1, P.weno.g2, P.weno.g3, P.weno.g12, P.weno.ig22, P.weno.ig3, P.weno.eps,
                         P.weno.sign_tol};
    for (int k = 0; k < 8; ++k) P.fweno[k] = float(w[k]);
    P.finv_dxi[0] = float(P.inv_dxi[0]);
    P.finv_dxi[1] = float(P.inv_dxi[1]);
    P.fca = float(P.ca);
    P.fcb = float(P.cb);
    P.fca_lo = float(P.ca - double(P.fca));
    P.fcb_lo = float(P.cb - double(P.fcb));
    P.fcst = float(P.cst);
    const size_t N = size_t(P.n1) * P.n2;
    if (P.fcs == 0) {
        P.fcs = N;
        P.fps = size_t(P.dim + 2) * N;
        P.fpsJ = N;
    }
}

cudaError_t launch_stage_fp64(const StageParams& P, cudaStream_t s);
cudaError_t launch_stage_mixed(const StageParams& P, cudaStream_t s);
// 2D tile shapes of the stage kernels (nodes BX x BY, NT threads >= the faces of either direction);
// the autotuner times each on the caller's problem
constexpr int STAGE_NTILES = 5;
void stage_tile_shape(bool mixed, int k, int* bx, int* by, int* nt);
// set the kernels' shared-memory attributes (call outside any stream capture)
cudaError_t stage_prepare_fp64(int dim);
cudaError_t stage_prepare_mixed(int dim);

// learned warm start (es_nn.cu): conv kernels' shared-memory attributes, weight copy, forward layer
cudaError_t nn_prepare();
cudaError_t nn_bf16_to_float(const uint16_t* w, float* f, size_t n, cudaStream_t s);
cudaError_t nn_conv_forward_f32(const float* in, const float* wf, const float* bias, float* out, int B, int Cin,
                                int Cout, int H, int W, int act, cudaStream_t s);
cudaError_t nn_conv_forward_bf16(const float* in, const uint16_t* w, const float* bias, float* out, int B, int Cin,
                                 int Cout, int H, int W, int act, cudaStream_t s);
// the same layer with bf16 [B][H][W][C] input and/or output (the context's inference buffers)
cudaError_t nn_conv_forward_bf16_fmt(const void* in, bool in_nhwc, const uint16_t* w, const float* bias, void* out,
                                     bool out_nhwc, int B, int Cin, int Cout, int H, int W, int act, cudaStream_t s);

}  // namespace es
