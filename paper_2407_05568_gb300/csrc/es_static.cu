// es_static.cu -- an SSP-RK3 step that allocates nothing (after its first call on a device).
//
// Some callers cannot call cudaMalloc at all: a solver embedded in a host
// application whose device memory is owned and budgeted by someone else, code
// that runs while a memory pool is being torn down or rebuilt, or a host
// process that must not add allocations after its start-up phase.  For them
// es_rk3_step_static advances (JU, J) by one SSP-RK3 step of the FP64 operator
// using only the arrays the caller passes plus a fixed scratch area that is
// compiled into this library: a file-scope __device__ array, set aside on every
// GPU that loads the library until the process exits.
//
// The scratch holds the two intermediate RK stage states and the device status
// word; it is sized for at most ES_STATIC_MAX_NODES mesh nodes.  All calls
// share it and it keeps the last call's contents, so calls whose work overlaps
// on the GPU (two streams, two host threads) race on it.
#include <cuda_runtime.h>
#include <mutex>
#include <string.h>

#include "es_internal.h"
#include "es_vdw.h"

using namespace es;

namespace {

constexpr int MAX_DEVICES = 64;
constexpr size_t STATUS_DOUBLES = 32;      // 256 bytes set aside for the status word
// two stage states of (dim + 2) + 1 fields (JU and J) for up to 2D meshes
constexpr size_t SCRATCH_DOUBLES = STATUS_DOUBLES + 2 * size_t(5) * ES_STATIC_MAX_NODES;

__device__ __align__(256) double g_static_scratch[SCRATCH_DOUBLES];

std::mutex g_setup_mutex;
double* g_scratch_ptr[MAX_DEVICES];
int g_prepared[MAX_DEVICES][3];            // stage kernel attributes set, per dim

// Device address of the scratch array on the current device (looked up once
// per device with that device current), and the stage kernel's shared-memory
// attribute for this dimension.  Under lazy module loading the symbol lookup is
// also what loads this library's modules, and with them the array.
int setup_current_device(int dim, double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return ES_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return ES_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    if (!g_prepared[dev][dim]) {
        if (stage_prepare_fp64(dim) != cudaSuccess) return ES_ERR_CUDA;
        g_prepared[dev][dim] = 1;
    }
    *out = g_scratch_ptr[dev];
    return ES_OK;
}

// the parameter checks of es_create that apply to this call (1D/2D, FP64, periodic or outflow ends)
bool params_ok(const es_params* p) {
    if (!p || (p->dim != 1 && p->dim != 2) || p->precision != ES_PREC_FP64) return false;
    if (p->n1 < 8 || (p->dim == 1 && p->n2 != 1) || (p->dim == 2 && p->n2 < 8)) return false;
    if (p->n3 != 0 && p->n3 != 1) return false;
    if (p->tile < 0 || p->tile > ES_NTILES) return false;
    if ((long long)p->n1 * p->n2 > ES_STATIC_MAX_NODES) return false;
    for (int k = 0; k < p->dim; ++k) {
        if (!(p->dxi[k] > 0.0)) return false;
        if (p->bc[k] != ES_BC_PERIODIC && p->bc[k] != ES_BC_OUTFLOW) return false;
        if (p->bc[k] == ES_BC_PERIODIC && !(p->period[k] > 0.0)) return false;
    }
    if (!(p->R > 0.0) || !(p->cv > 0.0) || !(p->a >= 0.0) || !(p->b >= 0.0)) return false;
    if (!(p->weno_gamma[0] > 0.0) || !(p->weno_gamma[1] > 0.0) || !(p->weno_gamma[2] > 0.0)) return false;
    if (!(p->weno_eps > 0.0) || !(p->sign_tol >= 0.0) || p->sign_tol > 1e-2) return false;
    return true;
}

}  // namespace

extern "C" int es_rk3_step_static(const es_params* p, double dt, double* JU, double* J, const double* x,
                                  const double* xdot, void* stream) {
    if (!params_ok(p) || !JU || !J || !x || !(dt >= 0.0)) return ES_ERR_ARG;
    double* scratch = nullptr;
    int rc = setup_current_device(p->dim, &scratch);
    if (rc != ES_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevStatus* status = reinterpret_cast<DevStatus*>(scratch);
    // the status word must start at zero; the stage buffers are written before they are read
    if (cudaMemsetAsync(status, 0, sizeof(DevStatus), s) != cudaSuccess) return ES_ERR_CUDA;

    const size_t N = size_t(p->n1) * p->n2;
    const int nc = p->dim + 2;
    double* S1 = scratch + STATUS_DOUBLES;
    double* S1J = S1 + nc * N;
    double* S2 = S1J + N;
    double* S2J = S2 + nc * N;

    StageParams P;
    memset(&P, 0, sizeof(P));
    P.dim = p->dim;
    P.n1 = p->n1;
    P.n2 = p->n2;
    P.bc[0] = p->bc[0];
    P.bc[1] = p->dim == 2 ? p->bc[1] : ES_BC_PERIODIC;
    P.inv_dxi[0] = 1.0 / p->dxi[0];
    P.inv_dxi[1] = p->dim == 2 ? 1.0 / p->dxi[1] : 0.0;
    P.period[0] = p->period[0];
    P.period[1] = p->period[1];
    P.gas.a = p->a;
    P.gas.b = p->b;
    P.gas.R = p->R;
    P.gas.cv = p->cv;
    P.gas.delta = p->R / p->cv;
    gas_reciprocals(P.gas);
    const double g1 = p->weno_gamma[0], g2 = p->weno_gamma[1], g3 = p->weno_gamma[2];
    const double gs = g1 + g2 + g3;
    P.weno.g1 = g1 / gs;
    P.weno.g2 = g2 / gs;
    P.weno.g3 = g3 / gs;
    P.weno.g12 = g1 / (g1 + g2);
    P.weno.ig22 = (g1 + g2) / g2;
    P.weno.ig3 = gs / g3;
    P.weno.eps = p->weno_eps;
    P.weno.sign_tol = p->sign_tol;
    P.diss = p->dissipation;
    P.tile = p->tile > 0 ? p->tile - 1 : 0;
    P.status = status;
    P.dt_host = dt;
    P.xn = x;
    P.xdot = xdot;
    const double A[3] = {0.0, 0.75, 1.0 / 3.0};
    const double B[3] = {1.0, 0.25, 2.0 / 3.0};
    const double C[3] = {0.0, 1.0, 0.5};
    const double* srcU[3] = {JU, S1, S2};
    const double* srcJ[3] = {J, S1J, S2J};
    double* dstU[3] = {S1, S2, JU};
    double* dstJ[3] = {S1J, S2J, J};
    for (int st = 0; st < 3; ++st) {
        P.ca = A[st];
        P.cb = B[st];
        P.cst = C[st];
        P.JUn = JU;
        P.Jn = J;
        P.JUs = srcU[st];
        P.Js = srcJ[st];
        P.JUo = dstU[st];
        P.Jo = dstJ[st];
        if (launch_stage_fp64(P, s) != cudaSuccess) return ES_ERR_CUDA;
    }
    DevStatus host_status = {0, 0};
    if (cudaMemcpyAsync(&host_status, status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return ES_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ES_ERR_CUDA;
    return host_status.code;
}
