// es_batch.h -- parameters of the batched persistent kernel (many 1D problems).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "es_df.cuh"
#include "es_internal.h"

namespace es {

struct BatchParams {
    int nprob;
    const int* order;             // queue order of the problems (longest first)
    const int* lengths;           // nodes per problem (>= 8)
    const long long* offsets;     // first node of each problem in the packed arrays
    size_t ntot;                  // total nodes
    // state (mixed form): JU [2][3][ntot], J [2][ntot] as (hi, lo) float planes
    float* JU;
    float* J;
    float* S1;
    float* S1J;
    float* S2;
    float* S2J;
    float* disp;                  // x_i - i/(L - 1), [ntot]
    float* xdot;                  // [ntot]
    float* work;                  // 9 scratch fields of ntot floats (monitor, filter, Jacobi)
    double* tprob;                // time of each problem
    int* queue;                   // work counter, zeroed before each launch
    int nsteps;
    double t_end;
    float cfl;
    int moving;
    int kappa;
    float w0, w1, w2;             // monitor weights
    int filter_passes, sweeps;
    StageParams tmpl;             // gas, WENO and the float constants of the stage kernel
    mixed::GasDF gdf;             // gas constants as (hi, lo) pairs for the monitor's G
};

// CTA shapes (threads per CTA) of the batched kernel; the autotuner times each
constexpr int BATCH_NSHAPES = 3;
extern const int BATCH_SHAPES[BATCH_NSHAPES];
cudaError_t batch_prepare();
cudaError_t batch_launch(const BatchParams& B, int grid, int bt, cudaStream_t s);
int batch_blocks_per_sm(int bt);
size_t batch_smem_bytes(int bt);

}  // namespace es
