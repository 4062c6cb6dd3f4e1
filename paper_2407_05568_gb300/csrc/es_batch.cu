// es_batch.cu -- many independent 1D problems in one persistent launch (mixed form).
//
// Each CTA takes a whole problem from an atomic work queue (problems ordered
// longest first) and advances it by `nsteps` full steps -- its own CFL time
// step (eq. cfl), its own mesh redistribution (Sec. 4: monitor with G, low-pass
// filter, Jacobi sweeps, limiter, mesh velocity) and the three SSP-RK3 stages,
// each stage a loop over 254-node chunks of the fused operator -- using only
// __syncthreads between phases.  No CTA ever waits for another, so there is no
// grid-wide synchronisation and no spin-wait.  The state of all problems is
// packed component-major: value c of node i of problem p at c * ntot + off_p + i.
//
// The mesh of a 1D problem on [0, 1] with L nodes is stored as the FP32
// displacement d_i = x_i - i/(L - 1) from the uniform computational mesh; the
// Jacobi sweeps and the limiter work on d directly (the uniform part cancels
// exactly), so the whole per-step pipeline runs on the FP32 pipe.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "es_batch.h"
#include "es_mixed_device.cuh"

namespace es {

using namespace mixed;

namespace {

// CTA shapes the autotuner chooses from: BT threads, chunks of BT - 2 nodes per stage tile
template <int BT>
struct BatchShape {
    static constexpr int BXC = BT - 2;
    using TB = TileF<1, BXC, 1, BT>;
    static constexpr int MIN_BLOCKS = BT >= 512 ? 1 : 768 / BT;     // 24 warps per SM (80 registers) below 512
};

__device__ __forceinline__ float block_max_f(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = red[0];
    for (int w = 1; w < int(blockDim.x) / 32; ++w) r = fmaxf(r, red[w]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ float block_min_f(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = red[0];
    for (int w = 1; w < int(blockDim.x) / 32; ++w) r = fminf(r, red[w]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ int clampi(int i, int L) { return i < 0 ? 0 : (i >= L ? L - 1 : i); }

template <int BT>
__global__ void __launch_bounds__(BT, BatchShape<BT>::MIN_BLOCKS) batch_kernel(BatchParams B) {
    constexpr int BXC = BatchShape<BT>::BXC;
    extern __shared__ float smemf[];
    __shared__ float red[BT / 32];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    const GasF G = gas_f(B.tmpl);
    const WenoF W = weno_f(B.tmpl);
    const size_t ntot = B.ntot;
    const float RK_A[3] = {0.0f, 0.75f, 1.0f / 3.0f};
    const float RK_B[3] = {1.0f, 0.25f, 2.0f / 3.0f};
    const float RK_C[3] = {0.0f, 1.0f, 0.5f};

    for (;;) {
        if (tid == 0) s_item = atomicAdd(B.queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= B.nprob) break;
        const int p = B.order[item];
        const int L = B.lengths[p];
        const size_t off = size_t(B.offsets[p]);
        const float dxi = 1.0f / float(L - 1);
        const float idxi = float(L - 1);
        float* d = B.disp + off;
        float* xd = B.xdot + off;
        float* rhoF = B.work + off;
        float* GF = B.work + ntot + off;
        float* t0 = B.work + 2 * ntot + off;
        float* t1 = B.work + 3 * ntot + off;
        float* t2 = B.work + 4 * ntot + off;
        float* om0 = B.work + 5 * ntot + off;
        float* om1 = B.work + 6 * ntot + off;
        float* da = B.work + 7 * ntot + off;
        float* db = B.work + 8 * ntot + off;
        double t = B.tprob[p];

        // node i's velocity, sound speed squared (rho, T for the monitor) and 1/J from the state
        auto node = [&](int i, float& rho, float& v, float& T, float& c2, float& iJ) {
            iJ = 1.0f / B.J[off + i];
            rho = B.JU[off + i] * iJ;
            v = B.JU[ntot + off + i] * iJ / rho;
            const float E = B.JU[2 * ntot + off + i] * iJ;
            T = (E / rho - 0.5f * v * v + G.a * rho) * G.icv;
            const float om = 1.0f - G.b * rho;
            c2 = (1.0f + G.delta) * G.R * T / (om * om) - 2.0f * G.a * rho;
        };
        for (int step = 0; step < B.nsteps; ++step) {
            // ---- time step, eq. cfl with the mesh at rest: dt = CFL / max (|v| + c) / (J dxi)
            float m = 0.0f;
            for (int i = tid; i < L; i += BT) {
                float rho, v, T, c2, iJ;
                node(i, rho, v, T, c2, iJ);
                const float lam = (fabsf(v) + sqrtf(fmaxf(c2, 0.0f))) * iJ * idxi;
                m = fmaxf(m, c2 > 0.0f ? lam : 3.0e38f);
                if (B.moving) {
                    // monitor fields: rho and the fundamental derivative G in double-float arithmetic from the
                    // (hi, lo) state planes (near the critical point p_nunu cancels to a small difference); the
                    // low parts wait in om0 / om1 (free until omega is formed) for the monitor's differences
                    const size_t q = off + i;
                    const df mom[1] = {{B.JU[ntot + q], B.JU[4 * ntot + q]}};
                    df r2, G2;
                    rho_G_df2({B.JU[q], B.JU[3 * ntot + q]}, mom, 1, {B.JU[2 * ntot + q], B.JU[5 * ntot + q]},
                              {B.J[q], B.J[ntot + q]}, B.gdf, &r2, &G2);
                    rhoF[i] = r2.hi;
                    om0[i] = r2.lo;
                    GF[i] = G2.hi;
                    om1[i] = G2.lo;
                }
            }
            m = block_max_f(m, red);
            double dt = double(B.cfl) / double(m);
            const double left = B.t_end - t;
            if (left <= 1e-14 * fmax(1.0, fabs(B.t_end))) break;
            if (dt > left) dt = left;
            float dtf = float(dt);

            // ---- mesh redistribution (Sec. 4) on the displacement
            if (B.moving) {
                float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f;
                for (int i = tid; i < L; i += BT) {
                    // differences of neighbours from the double-float fields (block_max_f's barriers above
                    // order the writes of the fields before these reads), then rounded
                    const int ip = clampi(i + 1, L), im = clampi(i - 1, L);
                    const df rp = {rhoF[ip], om0[ip]}, rm = {rhoF[im], om0[im]};
                    const df Gp = {GF[ip], om1[ip]}, G0 = {GF[i], om1[i]}, Gm = {GF[im], om1[im]};
                    const float gr = 0.5f * df_diff(rp, rm) * idxi;
                    const float gg = 0.5f * df_diff(Gp, Gm) * idxi;
                    const float lg = df_second_diff(Gp, G0, Gm) * idxi * idxi;
                    const float a0 = gr * gr, a1 = B.kappa >= 2 ? gg * gg : 0.0f, a2 = lg * lg;
                    t0[i] = a0;
                    t1[i] = a1;
                    t2[i] = a2;
                    m0 = fmaxf(m0, a0);
                    m1 = fmaxf(m1, a1);
                    m2 = fmaxf(m2, a2);
                }
                m0 = block_max_f(m0, red);
                m1 = block_max_f(m1, red);
                m2 = block_max_f(m2, red);
                const float c0 = m0 > 0.0f ? B.w0 / m0 : 0.0f;
                const float c1 = m1 > 0.0f ? B.w1 / m1 : 0.0f;
                const float c2 = m2 > 0.0f ? B.w2 / m2 : 0.0f;
                for (int i = tid; i < L; i += BT) om0[i] = sqrtf(1.0f + c0 * t0[i] + c1 * t1[i] + c2 * t2[i]);
                __syncthreads();
                float* om = om0;
                float* ot = om1;
                for (int f = 0; f < B.filter_passes; ++f) {
                    for (int i = tid; i < L; i += BT)
                        ot[i] = 0.25f * om[clampi(i - 1, L)] + 0.5f * om[i] + 0.25f * om[clampi(i + 1, L)];
                    __syncthreads();
                    float* tmp = om; om = ot; ot = tmp;
                }
                // Jacobi sweeps x_i <- (w+ x_{i+1} + w- x_{i-1})/(w+ + w-), written for the change
                // delta = x - x^n from the step's mesh: with a+- = w+-/(w+ + w-) and the constant part
                // g_i = a+ (x^n_{i+1} - x^n_i) + a- (x^n_{i-1} - x^n_i), formed once per solve from the
                // spacings (dxi + d_{i+1} - d_i),
                //   delta_i <- g_i + a+ delta_{i+1} + a- delta_{i-1},  delta = 0 at the fixed ends.
                // A sweep then rounds the small change, not the displacement d (up to a third of the
                // domain), and the mesh velocity needs no difference of two displacements.
                float* ap = t0;
                float* gc = t1;
                for (int i = tid; i < L; i += BT) {
                    if (i == 0 || i == L - 1) {
                        ap[i] = 0.0f;
                        gc[i] = 0.0f;
                    } else {
                        const float wp = 0.5f * (om[i] + om[i + 1]), wm = 0.5f * (om[i] + om[i - 1]);
                        const float a = wp / (wp + wm);
                        ap[i] = a;
                        gc[i] = a * (dxi + d[i + 1] - d[i]) - (1.0f - a) * (dxi + d[i] - d[i - 1]);
                    }
                    da[i] = 0.0f;
                }
                __syncthreads();
                const float* din = da;
                float* dout = db;
                for (int k = 0; k < B.sweeps; ++k) {
                    for (int i = tid; i < L; i += BT)
                        dout[i] = (i == 0 || i == L - 1)
                                      ? 0.0f
                                      : gc[i] + ap[i] * din[i + 1] + (1.0f - ap[i]) * din[i - 1];
                    __syncthreads();
                    din = dout;
                    dout = (dout == da) ? db : da;
                }
                // limiter: each node moves at most half of its spacing towards its neighbour
                float g = 1.0f;
                for (int i = tid; i < L; i += BT) {
                    const float del = din[i];
                    if (del < 0.0f && i > 0) g = fminf(g, -(dxi + d[i] - d[i - 1]) / (2.0f * del));
                    else if (del > 0.0f && i < L - 1) g = fminf(g, (dxi + d[i + 1] - d[i]) / (2.0f * del));
                }
                g = block_min_f(g, red);
                const float fv = g / dtf;
                for (int i = tid; i < L; i += BT) xd[i] = fv * din[i];
                // eq. cfl with this mesh velocity (J xi_t = -xdot): dt = min(dt, CFL / max (|v - xdot| + c) / (J dxi));
                // xdot keeps its value, so the mesh moves less than Delta_gamma allows
                float mv = 0.0f;
                for (int i = tid; i < L; i += BT) {
                    float rho, v, T, c2, iJ;
                    node(i, rho, v, T, c2, iJ);
                    const float lam = (fabsf(v - xd[i]) + sqrtf(fmaxf(c2, 0.0f))) * iJ * idxi;
                    mv = fmaxf(mv, c2 > 0.0f ? lam : 3.0e38f);
                }
                mv = block_max_f(mv, red);
                const double dtm = double(B.cfl) / double(mv);
                if (dtm < dt) {
                    dt = dtm;
                    dtf = float(dt);
                }
            }

            // ---- three fused RK stages, each a loop over BXC-node chunks
            StageParams P = B.tmpl;
            P.n1 = L;
            P.n2 = 1;
            P.inv_dxi[0] = double(idxi);
            P.finv_dxi[0] = idxi;
            P.fcs = ntot;
            P.fps = 3 * ntot;
            P.fpsJ = ntot;
            P.fdisp = d;
            P.fxdot = B.moving ? xd : nullptr;
            P.mode = 0;
            for (int st = 0; st < 3; ++st) {
                P.fca = RK_A[st];
                P.fcb = RK_B[st];
                P.fca_lo = st == 2 ? float(1.0 / 3.0 - double(RK_A[2])) : 0.0f;
                P.fcb_lo = st == 2 ? float(2.0 / 3.0 - double(RK_B[2])) : 0.0f;
                P.fcst = RK_C[st];
                P.fJUn = B.JU + off;
                P.fJn = B.J + off;
                P.fJUs = (st == 0 ? B.JU : (st == 1 ? B.S1 : B.S2)) + off;
                P.fJs = (st == 0 ? B.J : (st == 1 ? B.S1J : B.S2J)) + off;
                P.fJUo = (st == 0 ? B.S1 : (st == 1 ? B.S2 : B.JU)) + off;
                P.fJo = (st == 0 ? B.S1J : (st == 1 ? B.S2J : B.J)) + off;
                for (int c0 = 0; c0 < L; c0 += BXC) {
                    stage_tile_mixed<1, BXC, 1, BT>(smemf, P, c0, 0, dtf, G, W);
                    __syncthreads();
                }
            }
            if (B.moving)
                for (int i = tid; i < L; i += BT) d[i] += dtf * xd[i];
            __syncthreads();
            t += dt;
        }
        if (tid == 0) B.tprob[p] = t;
    }
}

template <int BT>
cudaError_t prepare_shape() {
    return cudaFuncSetAttribute(batch_kernel<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(BatchShape<BT>::TB::SMEM));
}

template <int BT>
int blocks_per_sm_shape() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<BT>, BT, BatchShape<BT>::TB::SMEM);
    return nb;
}

}  // namespace

const int BATCH_SHAPES[BATCH_NSHAPES] = {128, 256, 512};

size_t batch_smem_bytes(int bt) {
    return bt == 128 ? BatchShape<128>::TB::SMEM : bt == 512 ? BatchShape<512>::TB::SMEM : BatchShape<256>::TB::SMEM;
}

cudaError_t batch_prepare() {
    cudaError_t e = prepare_shape<128>();
    if (e == cudaSuccess) e = prepare_shape<256>();
    if (e == cudaSuccess) e = prepare_shape<512>();
    return e;
}

cudaError_t batch_launch(const BatchParams& B, int grid, int bt, cudaStream_t s) {
    switch (bt) {
        case 128: batch_kernel<128><<<grid, 128, BatchShape<128>::TB::SMEM, s>>>(B); break;
        case 512: batch_kernel<512><<<grid, 512, BatchShape<512>::TB::SMEM, s>>>(B); break;
        case 256: batch_kernel<256><<<grid, 256, BatchShape<256>::TB::SMEM, s>>>(B); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int batch_blocks_per_sm(int bt) {
    return bt == 128 ? blocks_per_sm_shape<128>() : bt == 512 ? blocks_per_sm_shape<512>() : blocks_per_sm_shape<256>();
}

// per-problem elementwise kernels (one CTA per problem)
__global__ void k_batch_set(BatchParams B, Gas Gd, const double* rho, const double* v, const double* pr) {
    const int p = blockIdx.x;
    const int L = B.lengths[p];
    const size_t off = size_t(B.offsets[p]);
    const size_t n = B.ntot;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const size_t id = off + i;
        const double r = rho[id], u = v[id];
        const double T = (pr[id] + Gd.a * r * r) * (1.0 - Gd.b * r) / (Gd.R * r);
        const double E = r * (Gd.cv * T - Gd.a * r) + 0.5 * r * u * u;
        const double vals[3] = {r, r * u, E};            // J = 1 on the uniform initial mesh
        for (int c = 0; c < 3; ++c) {
            const float hi = float(vals[c]);
            B.JU[c * n + id] = hi;
            B.JU[3 * n + c * n + id] = float(vals[c] - double(hi));
        }
        B.J[id] = 1.0f;
        B.J[n + id] = 0.0f;
        B.disp[id] = 0.0f;
        B.xdot[id] = 0.0f;
    }
    if (threadIdx.x == 0) B.tprob[p] = 0.0;
}

// conservative state, mesh and time of every problem: (JU, J) into (hi, lo) planes, x into the displacement
// from the uniform mesh, the mesh velocity cleared
__global__ void k_batch_set_state(BatchParams B, const double* JU, const double* J, const double* x,
                                  const double* t) {
    const int p = blockIdx.x;
    const int L = B.lengths[p];
    const size_t off = size_t(B.offsets[p]);
    const size_t n = B.ntot;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const size_t id = off + i;
        for (int c = 0; c < 3; ++c) {
            const double v = JU[c * n + id];
            const float hi = float(v);
            B.JU[c * n + id] = hi;
            B.JU[3 * n + c * n + id] = float(v - double(hi));
        }
        const float jh = float(J[id]);
        B.J[id] = jh;
        B.J[n + id] = float(J[id] - double(jh));
        B.disp[id] = float(x[id] - double(i) / double(L - 1));
        B.xdot[id] = 0.0f;
    }
    if (threadIdx.x == 0) B.tprob[p] = t[p];
}

__global__ void k_batch_get(BatchParams B, double* JU, double* J, double* x, double* t) {
    const int p = blockIdx.x;
    const int L = B.lengths[p];
    const size_t off = size_t(B.offsets[p]);
    const size_t n = B.ntot;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const size_t id = off + i;
        for (int c = 0; c < 3; ++c) JU[c * n + id] = double(B.JU[c * n + id]) + double(B.JU[3 * n + c * n + id]);
        J[id] = double(B.J[id]) + double(B.J[n + id]);
        x[id] = double(i) / double(L - 1) + double(B.disp[id]);
    }
    if (threadIdx.x == 0 && t) t[p] = B.tprob[p];
}

}  // namespace es

// ------------------------------------------------------------------ C ABI
using namespace es;

struct es_batch {
    es_params p;
    cudaStream_t stream, cap_stream;
    BatchParams B;
    int* d_order;
    int* d_lengths;
    long long* d_offsets;
    float* state;
    float* work;
    double* tprob;
    int* queue;
    DevStatus* status;
    int grid;
    int bt;                           // threads per CTA (the CTA shape)
    int nsm;
    cudaGraphExec_t gexec;
    int g_nsteps;
    double g_tend;
    char msg[256];
};

namespace {

int bfail(es_batch* b, cudaError_t e, const char* where) {
    if (b) snprintf(b->msg, sizeof(b->msg), "%s: %s", where, cudaGetErrorString(e));
    return ES_ERR_CUDA;
}

#define BCK(call, where)                               \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return bfail(b, e_, where); \
    } while (0)

// CTA shape and the persistent grid: SMs x resident CTAs of that shape, at most one per problem
void set_shape(es_batch* b, int bt) {
    b->bt = bt;
    const int per_sm = batch_blocks_per_sm(bt);
    b->grid = b->nsm * (per_sm > 0 ? per_sm : 1);
    if (b->grid > b->B.nprob) b->grid = b->B.nprob;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
}

}  // namespace

extern "C" {

int es_batch_create(es_batch** out, const es_params* p, int nprob, const int* lengths_host, void* stream) {
    if (!out || !p || !lengths_host || nprob <= 0) return ES_ERR_ARG;
    *out = nullptr;
    if (p->dim != 1 || p->precision != ES_PREC_MIXED || !(p->cfl > 0.0) || !(p->R > 0.0) || !(p->cv > 0.0) ||
        !(p->weno_eps > 0.0) || p->filter_passes < 0 || p->jacobi_sweeps < 0 || p->jacobi_sweeps > 100000 ||
        (p->moving && (p->monitor != ES_MONITOR_VDW || p->kappa < 1 || p->kappa > 2)))
        return ES_ERR_ARG;
    long long ntot = 0;
    for (int k = 0; k < nprob; ++k) {
        if (lengths_host[k] < 8 || lengths_host[k] > (1 << 24)) return ES_ERR_ARG;
        ntot += lengths_host[k];
    }
    if (ntot > (1LL << 31)) return ES_ERR_ARG;
    es_batch* b = (es_batch*)calloc(1, sizeof(es_batch));
    if (!b) return ES_ERR_ARG;
    b->p = *p;
    b->stream = (cudaStream_t)stream;
    // host-side queue order: longest problems first (a greedy longest-processing-time schedule)
    int* order = (int*)malloc(sizeof(int) * nprob);
    long long* offs = (long long*)malloc(sizeof(long long) * nprob);
    long long acc = 0;
    for (int k = 0; k < nprob; ++k) {
        order[k] = k;
        offs[k] = acc;
        acc += lengths_host[k];
    }
    for (int a = 1; a < nprob; ++a) {                   // insertion sort by length, descending
        int v = order[a], j = a - 1;
        while (j >= 0 && lengths_host[order[j]] < lengths_host[v]) { order[j + 1] = order[j]; --j; }
        order[j + 1] = v;
    }
    const size_t n = size_t(ntot);
    int rc = ES_OK;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMalloc((void**)&b->d_order, sizeof(int) * nprob))) break;
        if ((e = cudaMalloc((void**)&b->d_lengths, sizeof(int) * nprob))) break;
        if ((e = cudaMalloc((void**)&b->d_offsets, sizeof(long long) * nprob))) break;
        // state planes: JU 6n, J 2n, S1 6n, S1J 2n, S2 6n, S2J 2n, disp n, xdot n
        if ((e = cudaMalloc((void**)&b->state, sizeof(float) * n * 26))) break;
        if ((e = cudaMalloc((void**)&b->work, sizeof(float) * n * 9))) break;
        if ((e = cudaMalloc((void**)&b->tprob, sizeof(double) * nprob))) break;
        if ((e = cudaMalloc((void**)&b->queue, sizeof(int)))) break;
        if ((e = cudaMalloc((void**)&b->status, sizeof(DevStatus)))) break;
        if ((e = cudaMemcpy(b->d_order, order, sizeof(int) * nprob, cudaMemcpyHostToDevice))) break;
        if ((e = cudaMemcpy(b->d_lengths, lengths_host, sizeof(int) * nprob, cudaMemcpyHostToDevice))) break;
        if ((e = cudaMemcpy(b->d_offsets, offs, sizeof(long long) * nprob, cudaMemcpyHostToDevice))) break;
        if ((e = cudaMemset(b->status, 0, sizeof(DevStatus)))) break;
        if ((e = cudaMemset(b->tprob, 0, sizeof(double) * nprob))) break;
        if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking))) break;
        if ((e = batch_prepare())) break;
    } while (0);
    free(order);
    free(offs);
    if (e != cudaSuccess) {
        rc = bfail(b, e, "es_batch_create");
        es_batch_destroy(b);
        return rc;
    }
    BatchParams& B = b->B;
    B.nprob = nprob;
    B.order = b->d_order;
    B.lengths = b->d_lengths;
    B.offsets = b->d_offsets;
    B.ntot = n;
    B.JU = b->state;
    B.J = b->state + 6 * n;
    B.S1 = b->state + 8 * n;
    B.S1J = b->state + 14 * n;
    B.S2 = b->state + 16 * n;
    B.S2J = b->state + 22 * n;
    B.disp = b->state + 24 * n;
    B.xdot = b->state + 25 * n;
    B.work = b->work;
    B.tprob = b->tprob;
    B.queue = b->queue;
    B.cfl = float(p->cfl);
    B.gdf = mixed::gas_df(p->a, p->b, p->R, p->cv);
    B.moving = p->moving;
    B.kappa = p->kappa;
    B.w0 = float(p->alpha[0]);
    B.w1 = float(p->kappa >= 2 ? p->alpha[1] : 0.0);
    B.w2 = float(p->alpha[p->kappa]);
    B.filter_passes = p->filter_passes;
    B.sweeps = p->jacobi_sweeps;
    StageParams& P = B.tmpl;
    memset(&P, 0, sizeof(P));
    P.dim = 1;
    P.bc[0] = ES_BC_OUTFLOW;
    P.bc[1] = ES_BC_PERIODIC;
    P.gas.a = p->a;
    P.gas.b = p->b;
    P.gas.R = p->R;
    P.gas.cv = p->cv;
    P.gas.delta = p->R / p->cv;
    gas_reciprocals(P.gas);
    const double g1 = p->weno_gamma[0], g2 = p->weno_gamma[1], g3 = p->weno_gamma[2], gs = g1 + g2 + g3;
    P.weno.g1 = g1 / gs;
    P.weno.g2 = g2 / gs;
    P.weno.g3 = g3 / gs;
    P.weno.g12 = g1 / (g1 + g2);
    P.weno.ig22 = (g1 + g2) / g2;
    P.weno.ig3 = gs / g3;
    P.weno.eps = p->weno_eps;
    P.weno.sign_tol = p->sign_tol;
    P.diss = p->dissipation;
    P.status = b->status;
    P.n1 = 8;
    P.n2 = 1;
    P.fcs = n;                                         // the kernel sets the per-problem fields
    set_float_params(P);
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    b->nsm = nsm;
    set_shape(b, 256);
    *out = b;
    return ES_OK;
}

void es_batch_destroy(es_batch* b) {
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    void* bufs[] = {b->d_order, b->d_lengths, b->d_offsets, b->state, b->work, b->tprob, b->queue, b->status};
    for (void* q : bufs)
        if (q) cudaFree(q);
    free(b);
}

int64_t es_batch_nodes(es_batch* b) { return b ? (int64_t)b->B.ntot : 0; }

int es_batch_set_prim(es_batch* b, const double* rho, const double* v, const double* pr) {
    if (!b || !rho || !v || !pr) return ES_ERR_ARG;
    Gas Gd;
    Gd.a = b->p.a;
    Gd.b = b->p.b;
    Gd.R = b->p.R;
    Gd.cv = b->p.cv;
    Gd.delta = b->p.R / b->p.cv;
    gas_reciprocals(Gd);
    k_batch_set<<<b->B.nprob, 256, 0, b->stream>>>(b->B, Gd, rho, v, pr);
    BCK(cudaGetLastError(), "k_batch_set");
    return ES_OK;
}

int es_batch_set_state(es_batch* b, const double* JU, const double* J, const double* x, const double* t) {
    if (!b || !JU || !J || !x || !t) return ES_ERR_ARG;
    k_batch_set_state<<<b->B.nprob, 256, 0, b->stream>>>(b->B, JU, J, x, t);
    BCK(cudaGetLastError(), "k_batch_set_state");
    return ES_OK;
}

int es_batch_steps(es_batch* b, int nsteps, double t_end) {
    if (!b || nsteps < 0) return ES_ERR_ARG;
    if (nsteps == 0) return ES_OK;
    if (!b->gexec || b->g_nsteps != nsteps || b->g_tend != t_end) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        BatchParams B = b->B;
        B.nsteps = nsteps;
        B.t_end = t_end;
        cudaGraph_t graph;
        BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e1 = cudaMemsetAsync(b->queue, 0, sizeof(int), b->cap_stream);
        cudaError_t e2 = batch_launch(B, b->grid, b->bt, b->cap_stream);
        cudaError_t e3 = cudaStreamEndCapture(b->cap_stream, &graph);
        if (e1 != cudaSuccess) return bfail(b, e1, "memset");
        if (e2 != cudaSuccess) return bfail(b, e2, "batch kernel");
        if (e3 != cudaSuccess) return bfail(b, e3, "end capture");
        cudaError_t e = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(b, e, "instantiate");
        b->g_nsteps = nsteps;
        b->g_tend = t_end;
    }
    BCK(cudaGraphLaunch(b->gexec, b->stream), "graph launch");
    return ES_OK;
}

int es_batch_autotune(es_batch* b, int* bt_host, double* ms_host) {
    if (!b) return ES_ERR_ARG;
    const size_t sbytes = sizeof(float) * b->B.ntot * 26, tbytes = sizeof(double) * b->B.nprob;
    char* save = nullptr;
    BCK(cudaMalloc((void**)&save, sbytes + tbytes), "cudaMalloc");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(save, b->state, sbytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(save + sbytes, b->tprob, tbytes, cudaMemcpyDeviceToDevice, b->stream);
    BatchParams B = b->B;
    B.nsteps = 1;
    B.t_end = 1e300;
    int best = 256;
    float best_ms = 3.0e38f;
    for (int k = 0; k < BATCH_NSHAPES && e == cudaSuccess; ++k) {
        const int bt = BATCH_SHAPES[k];
        const int per_sm = batch_blocks_per_sm(bt);
        int grid = b->nsm * (per_sm > 0 ? per_sm : 1);
        if (grid > b->B.nprob) grid = b->B.nprob;
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run loads the kernel
            e = cudaMemcpyAsync(b->state, save, sbytes, cudaMemcpyDeviceToDevice, b->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(b->tprob, save + sbytes, tbytes, cudaMemcpyDeviceToDevice, b->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(b->queue, 0, sizeof(int), b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess) e = batch_launch(B, grid, bt, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        }
        if (ms_host) ms_host[k] = ms;
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = bt;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->state, save, sbytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->tprob, save + sbytes, tbytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    if (e != cudaSuccess) return bfail(b, e, "autotune");
    set_shape(b, best);
    if (bt_host) *bt_host = best;
    return ES_OK;
}

int es_batch_get(es_batch* b, double* JU, double* J, double* x, double* t) {
    if (!b || !JU || !J || !x) return ES_ERR_ARG;
    k_batch_get<<<b->B.nprob, 256, 0, b->stream>>>(b->B, JU, J, x, t);
    BCK(cudaGetLastError(), "k_batch_get");
    return ES_OK;
}

int es_batch_check(es_batch* b) {
    if (!b) return ES_ERR_ARG;
    BCK(cudaStreamSynchronize(b->stream), "sync");
    DevStatus h = {0, 0};
    BCK(cudaMemcpy(&h, b->status, sizeof(h), cudaMemcpyDeviceToHost), "status");
    if (h.code) {
        snprintf(b->msg, sizeof(b->msg), "device status %d at node %d", h.code, h.index);
        DevStatus z = {0, 0};
        BCK(cudaMemcpy(b->status, &z, sizeof(z), cudaMemcpyHostToDevice), "clear status");
    }
    return h.code;
}

int es_batch_last_error(es_batch* b, char* buf, int len) {
    if (!b || !buf || len <= 0) return ES_ERR_ARG;
    snprintf(buf, len, "%s", b->msg);
    return ES_OK;
}

}  // extern "C"
