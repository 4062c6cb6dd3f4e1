// es_probe.cu -- the FP64 and FP32 arithmetic rates of the GPU the library runs on, measured.
//
// The stage kernels are bound by the FP64 pipe (plain form) or the FP32 pipe (mixed and batched
// forms), so their roofline denominators are these rates rather than nominal figures.  The probe
// runs a grid of SMs x 8 CTAs x 256 threads; every thread carries 8 independent chains of dependent
// fused multiply-adds a <- a b + c (enough independent work to fill the pipe), times the launch with
// CUDA events and keeps the best of several launches.  An FMA counts as two operations.
#include <cuda_runtime.h>

#include "es_vdw.h"

namespace {

constexpr int CHAINS = 8;
constexpr int UNROLL = 16;

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(T b, T c, int iters, T* sink) {
    T a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < UNROLL; ++r)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == T(-12345.0)) sink[blockIdx.x] = s;     // never true for these inputs; keeps the chains live
}

template <class T>
int measure(int iters, cudaStream_t s, double* tflops) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return ES_ERR_CUDA;
    const int grid = nsm * 8, block = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return ES_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ES_ERR_CUDA;
    }
    T* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(T) * grid) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return ES_ERR_CUDA;
    }
    const T b = T(0.999999), c = T(1e-6);
    float best = 1e30f;
    int rc = ES_OK;
    for (int rep = 0; rep < 6 && rc == ES_OK; ++rep) {           // the first launch warms up
        cudaEventRecord(e0, s);
        k_fma_chains<T><<<grid, block, 0, s>>>(b, c, iters, sink);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = ES_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != ES_OK) return rc;
    const double ops = 2.0 * double(grid) * block * CHAINS * UNROLL * double(iters);
    *tflops = ops / (double(best) * 1e-3) / 1e12;
    return ES_OK;
}

}  // namespace

extern "C" int es_selftest_peaks(double* fp64_tflops, double* fp32_tflops, void* stream) {
    if (!fp64_tflops || !fp32_tflops) return ES_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = measure<double>(64, s, fp64_tflops);               // ~5 ms per launch at ~1 TFLOP/s
    if (rc == ES_OK) rc = measure<float>(4096, s, fp32_tflops);  // ~5 ms per launch at ~80 TFLOP/s
    return rc;
}
