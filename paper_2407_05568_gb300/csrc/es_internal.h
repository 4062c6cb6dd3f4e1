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
};

cudaError_t launch_stage_fp64(const StageParams& P, cudaStream_t s);
cudaError_t launch_stage_mixed(const StageParams& P, cudaStream_t s);
// set the kernels' shared-memory attributes (call outside any stream capture)
cudaError_t stage_prepare_fp64(int dim);
cudaError_t stage_prepare_mixed(int dim);

}  // namespace es
