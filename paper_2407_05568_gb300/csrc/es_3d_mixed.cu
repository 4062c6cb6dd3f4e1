// es_3d_mixed.cu -- the mixed-precision form of the 3D path: the direction kernels on the FP32 pipe.
//
// As in the 1D/2D mixed form, the state is kept as double-float pairs (hi + lo float planes), the
// primitive state rho, v, T of every node carries a low part so that jumps between neighbours
// keep their digits, the two-point fluxes and MR-WENO5 run in float, and the dissipation works on
// entropy-variable jumps from the jump decomposition of Sec. 3.1 (eq. jumpV) shared by the faces
// of a line.  The node fields are computed once per node in double-float arithmetic and stored
// as floats (with the low parts), and the metrics are the FP64 cross-form metrics of es_3d.cu
// rounded to float at load.  The right-hand sides are accumulated over the
// three directions in float and the Shu-Osher combination is done in double-float.
#include <cuda.h>            // CUtensorMap (the encoder is fetched from the driver at run time)
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "es_3d.h"
#include "es_bits.cuh"
#include "es_3d_grid.cuh"
#include "es_device.cuh"
#include "es_internal.h"
#include "es_mesh_f32.h"
#include "es_mixed_device.cuh"

namespace es {
namespace mixed3 {

using mixed::df;
using mixed::df_add;
using mixed::df_add_f;
using mixed::df_diff;
using mixed::df_second_diff;
using mixed::df_mul;
using mixed::df_mul_f;
using mixed::df_recip;
using mixed::GasF;
using mixed::inv_log_mean_f;
using mixed::inv_log_mean_j;
using mixed::mr_weno5_f;
using mixed::WenoF;

// float node fields (global planes and shared-memory slots)
enum FieldM {
    M_RHO, M_V1, M_V2, M_V3, M_T, M_IT, M_OM, M_IOM, M_G, M_RT, M_VT1, M_VT2, M_VT3, M_V2T,
    M_RV1, M_RV2, M_RV3, M_RP, M_RHOL, M_V1L, M_V2L, M_V3L, M_TL,
    MF_COUNT,
    M_NX = MF_COUNT, M_NY, M_NZ, M_XT,
    MS_COUNT
};
static_assert(MF_COUNT <= 23, "the float node fields reuse the FP64 node-field buffer");

// ---------------------------------------------------------------- node fields
// From the double-float state (JU: hi plane [5][N] then lo plane; J: hi then lo) in double-float
// arithmetic on the FP32 pipe (as the 2D mixed tile does), stored as floats with the low parts of
// rho, v, T.
__global__ void k3_nodes_f(Grid3 g, GasF G, const float* JU, const float* J, float* NF, DevStatus* st) {
    const int N = g.n[0] * g.n[1] * g.n[2];
    const size_t P = size_t(N), LO = 5 * P;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const df iJ = df_recip({J[id], J[P + id]});
        const df rho = df_mul({JU[id], JU[LO + id]}, iJ);
        const df E = df_mul({JU[4 * P + id], JU[LO + 4 * P + id]}, iJ);
        const df irho = df_recip(rho);
        df m[3], v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            m[c] = df_mul({JU[(1 + c) * P + id], JU[LO + (1 + c) * P + id]}, iJ);
            v[c] = df_mul(m[c], irho);
        }
        const df ke = df_mul_f(df_add(df_add(df_mul(v[0], v[0]), df_mul(v[1], v[1])), df_mul(v[2], v[2])), 0.5f);
        // T = (E/rho - |v|^2/2 + a rho) / cv
        const df e = df_add(df_mul(E, irho), {-ke.hi, -ke.lo});
        const df Td = df_mul_f(df_add(e, df_mul_f(rho, G.a)), G.icv);
        const float r = rho.hi, Tf = Td.hi;
        const float om = 1.0f - G.b * r;
        const float iom = 1.0f / om;
        const float iT = 1.0f / Tf;
        const float p = r * G.R * Tf * iom - G.a * r * r;
        if (!(r > 0.0f) || !(om > 0.0f) || !(Tf > 0.0f) || !(p > 0.0f)) raise_error(st, ES_ERR_INADMISSIBLE, id);
        NF[M_RHO * P + id] = r;
        NF[M_RHOL * P + id] = rho.lo;
        NF[M_T * P + id] = Tf;
        NF[M_TL * P + id] = Td.lo;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            NF[(M_V1 + c) * P + id] = v[c].hi;
            NF[(M_V1L + c) * P + id] = v[c].lo;
            NF[(M_VT1 + c) * P + id] = v[c].hi * iT;
            NF[(M_RV1 + c) * P + id] = m[c].hi;
        }
        NF[M_IT * P + id] = iT;
        NF[M_OM * P + id] = om;
        NF[M_IOM * P + id] = iom;
        NF[M_G * P + id] = G.R * iom - G.a * r * iT;
        NF[M_RT * P + id] = r * iT;
        NF[M_V2T * P + id] = 2.0f * ke.hi * iT;
        NF[M_RP * P + id] = r / p;
    }
}

// ---------------------------------------------------------------- pair flux
__device__ __forceinline__ void pair_flux3_f(const float* S, int NB, int l, int r, float nx, float ny, float nz,
                                             float xt, const GasF& G, float* out) {
    const float rl = S[M_RHO * NB + l], rr = S[M_RHO * NB + r];
    const float Tl = S[M_T * NB + l], Tr = S[M_T * NB + r];
    const float rho_m = 0.5f * (rl + rr);
    const float T_m = 0.5f * (Tl + Tr);
    const float iT_m = 0.5f * (S[M_IT * NB + l] + S[M_IT * NB + r]);
    const float drho = (rl - rr) + (S[M_RHOL * NB + l] - S[M_RHOL * NB + r]);
    const float ilr = inv_log_mean_j(rl, rr, drho);
    const float ilT = inv_log_mean_j(Tl, Tr, (Tl - Tr) + (S[M_TL * NB + l] - S[M_TL * NB + r]));
    const float Pinv = S[M_IOM * NB + l] * S[M_IOM * NB + r];
    const float iTa = 1.0f / T_m;
    const float coef = G.Rb * Pinv - G.a * iTa;
    float D = G.R * ilr + coef - G.a * iTa;
    if (G.b > 0.0f) D += G.Rb * inv_log_mean_j(S[M_OM * NB + l], S[M_OM * NB + r], -G.b * drho);
    const float iD = 1.0f / D;
    const float g_m = 0.5f * (S[M_G * NB + l] + S[M_G * NB + r]);
    const float rT_m = 0.5f * (S[M_RT * NB + l] + S[M_RT * NB + r]);
    const float v2T_m = 0.5f * (S[M_V2T * NB + l] + S[M_V2T * NB + r]);
    float vm[3], vT[3], rv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        vm[c] = 0.5f * (S[(M_V1 + c) * NB + l] + S[(M_V1 + c) * NB + r]);
        vT[c] = 0.5f * (S[(M_VT1 + c) * NB + l] + S[(M_VT1 + c) * NB + r]);
        rv[c] = 0.5f * (S[(M_RV1 + c) * NB + l] + S[(M_RV1 + c) * NB + r]);
    }
    const float U1 = (rho_m * coef + g_m) * iD;
    const float F11 = (rv[0] * coef + g_m * vm[0]) * iD;
    const float F21 = (rv[1] * coef + g_m * vm[1]) * iD;
    const float F31 = (rv[2] * coef + g_m * vm[2]) * iD;
    const float P = rho_m * T_m * g_m;
    const float B0 = 0.5f * v2T_m - G.cv * T_m * ilT + 2.0f * G.a * rT_m;
    const float Q1 = xt * U1 + nx * F11 + ny * F21 + nz * F31;
    const float sv = vT[0] * vm[0] + vT[1] * vm[1] + vT[2] * vm[2];
    out[0] = Q1;
    out[1] = vm[0] * Q1 + nx * P;
    out[2] = vm[1] * Q1 + ny * P;
    out[3] = vm[2] * Q1 + nz * P;
    out[4] = (G.a * rT_m * (xt * rho_m + nx * rv[0] + ny * rv[1] + nz * rv[2]) + (sv - B0) * Q1 +
              P * (nx * vT[0] + ny * vT[1] + nz * vT[2])) /
             iT_m;
}

// entropy-variable jump V_j - V_i by eq. jumpV in general units (the 2D form of the mixed
// kernels with three velocity components)
__device__ __forceinline__ void entropy_jump3_f(const float* S, int NB, int i, int j, const GasF& G, float* dV) {
    const float ri = S[M_RHO * NB + i], rj = S[M_RHO * NB + j];
    const float Ti = S[M_T * NB + i], Tj = S[M_T * NB + j];
    const float dr = (rj - ri) + (S[M_RHOL * NB + j] - S[M_RHOL * NB + i]);
    const float dT = (Tj - Ti) + (S[M_TL * NB + j] - S[M_TL * NB + i]);
    const float iTa = 2.0f / (Ti + Tj);
    float crho = G.R * inv_log_mean_j(ri, rj, -dr) + G.Rb * S[M_IOM * NB + i] * S[M_IOM * NB + j] - 2.0f * G.a * iTa;
    if (G.b > 0.0f) crho += G.Rb * inv_log_mean_j(S[M_OM * NB + i], S[M_OM * NB + j], G.b * dr);
    const float rT = 0.5f * (S[M_RT * NB + i] + S[M_RT * NB + j]);
    const float v2T = 0.5f * (S[M_V2T * NB + i] + S[M_V2T * NB + j]);
    const float cT = -G.cv * inv_log_mean_j(Ti, Tj, -dT) + (2.0f * G.a * rT + 0.5f * v2T) * iTa;
    float kin = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float vi = S[(M_V1 + c) * NB + i], vj = S[(M_V1 + c) * NB + j];
        const float dv = (vj - vi) + (S[(M_V1L + c) * NB + j] - S[(M_V1L + c) * NB + i]);
        kin += 0.5f * (vi + vj) * dv;
        dV[1 + c] = (dv - 0.5f * (S[(M_VT1 + c) * NB + i] + S[(M_VT1 + c) * NB + j]) * dT) * iTa;
    }
    dV[0] = dr * crho + dT * cT - kin * iTa;
    dV[4] = dT * S[M_IT * NB + i] * S[M_IT * NB + j];
}

// -1/2 Lambda T^{-1} R Y [[W]]^WENO at the face between l and l+1 with the 3D frame (as in the FP64
// 3D kernel), W measured from node l through the shared neighbour jumps JB (line offset jq)
__device__ __forceinline__ void face_dissipation3_f(const float* S, int NB, int l, float nx, float ny, float nz,
                                                    float xtf, const GasF& G, const WenoF& Wc, float* out,
                                                    DevStatus* st, const float* JB, int NJ, int jq) {
    const int r = l + 1;
    const float ilr = inv_log_mean_f(S[M_RHO * NB + l], S[M_RHO * NB + r]);
    const float rho = 1.0f / ilr;
    const float ilrp = inv_log_mean_f(S[M_RP * NB + l], S[M_RP * NB + r]);
    const float p = rho * ilrp;
    const float om = 1.0f - G.b * rho;
    const float T = (p + G.a * rho * rho) * om * ilr * G.iR;
    const float iom = 1.0f / om;
    const float c2 = (1.0f + G.delta) * G.R * T * iom * iom - 2.0f * G.a * rho;
    const float dcrit = G.R * T - 2.0f * G.a * rho * om * om;
    if (!(c2 > 0.0f) || !(dcrit > 0.0f) || !(om > 0.0f)) raise_error(st, ES_ERR_INADMISSIBLE, 0);
    const float c = sqrtf(c2);
    const float vm1 = 0.5f * (S[M_V1 * NB + l] + S[M_V1 * NB + r]);
    const float vm2 = 0.5f * (S[M_V2 * NB + l] + S[M_V2 * NB + r]);
    const float vm3 = 0.5f * (S[M_V3 * NB + l] + S[M_V3 * NB + r]);
    const float L = sqrtf(nx * nx + ny * ny + nz * nz);
    const float r12 = sqrtf(nx * nx + ny * ny);
    float ct = 1.0f, sn = 0.0f;
    if (r12 > 1e-12f * L) {                  // below: the rounding of metrics that vanish exactly
        const float ir = 1.0f / r12;
        ct = nx * ir;
        sn = ny * ir;
    }
    const float iL = 1.0f / L;
    const float cp = r12 * iL, sp = nz * iL;
    const float en[3] = {cp * ct, cp * sn, sp};
    const float et1[3] = {-sn, ct, 0.0f};
    const float et2[3] = {-sp * ct, -sp * sn, cp};
    const float vn = en[0] * vm1 + en[1] * vm2 + en[2] * vm3;
    const float vt1 = et1[0] * vm1 + et1[1] * vm2;
    const float vt2 = et2[0] * vm1 + et2[1] * vm2 + et2[2] * vm3;
    const float E = rho * (G.cv * T - G.a * rho) + 0.5f * rho * (vn * vn + vt1 * vt1 + vt2 * vt2);
    const float H = (E + p) * ilr;
    const float mid = H - c2 * om * G.idelta;
    const float ic2 = 1.0f / c2;
    const float sA = sqrtf(0.5f * rho * T * ic2);
    const float sE = sqrtf(G.R * G.delta * rho * T * T * ic2 / dcrit);
    const float sT = sqrtf(rho * T);
    const float Lam = fabsf(xtf + L * vn) + L * c;
    const float Hm = H - vn * c, Hp = H + vn * c;

    // V_j - V_l at nodes l-2 .. l+3 from the neighbour jumps (zero at l)
    float W[6][5];
    float cum[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        W[2][m] = 0.0f;
        cum[m] = 0.0f;
    }
#pragma unroll
    for (int o = 3; o < 6; ++o)
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            cum[m] += JB[m * NJ + jq + (o - 3)];
            W[o][m] = cum[m];
        }
#pragma unroll
    for (int m = 0; m < 5; ++m) cum[m] = 0.0f;
#pragma unroll
    for (int o = 1; o >= 0; --o)
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            cum[m] -= JB[m * NJ + jq + (o - 2)];
            W[o][m] = cum[m];
        }
    float aTV[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        if (o == 2) continue;
        const float V0 = W[o][0], V4 = W[o][4];
        const float a1 = W[o][1], a2 = W[o][2], a3 = W[o][3];
        const float V1 = en[0] * a1 + en[1] * a2 + en[2] * a3;
        const float V2 = et1[0] * a1 + et1[1] * a2;
        const float V3 = et2[0] * a1 + et2[1] * a2 + et2[2] * a3;
        const float base = V0 + vt1 * V2 + vt2 * V3;
        W[o][0] = sA * (base + (vn - c) * V1 + Hm * V4);
        W[o][1] = sE * (base + vn * V1 + mid * V4);
        W[o][2] = sT * (V2 + vt1 * V4);
        W[o][3] = sT * (V3 + vt2 * V4);
        W[o][4] = sA * (base + (vn + c) * V1 + Hp * V4);
        if (o == 3) {
            aTV[0] = fabsf(V0);
            aTV[1] = fabsf(V1);
            aTV[2] = fabsf(V2);
            aTV[3] = fabsf(V3);
            aTV[4] = fabsf(V4);
        }
    }
    const float avt1 = fabsf(vt1), avt2 = fabsf(vt2);
    const float common = aTV[0] + avt1 * aTV[2] + avt2 * aTV[3];
    float scl[5];
    scl[0] = sA * (common + fabsf(vn - c) * aTV[1] + fabsf(Hm) * aTV[4]);
    scl[1] = sE * (common + fabsf(vn) * aTV[1] + fabsf(mid) * aTV[4]);
    scl[2] = sT * (aTV[2] + (avt1 + c) * aTV[4]);
    scl[3] = sT * (aTV[3] + (avt2 + c) * aTV[4]);
    scl[4] = sA * (common + fabsf(vn + c) * aTV[1] + fabsf(Hp) * aTV[4]);
    float y[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const float wmin = mr_weno5_f(W[0][m], W[1][m], W[2][m], W[3][m], W[4][m], Wc);
        const float wplu = mr_weno5_f(W[5][m], W[4][m], W[3][m], W[2][m], W[1][m], Wc);
        const float jw = wplu - wmin;
        float j = W[3][m];
        if (fabsf(j) <= Wc.sign_tol * scl[m]) j = 0.0f;
        const bool keep = (jw > 0.0f && j > 0.0f) || (jw < 0.0f && j < 0.0f);
        y[m] = keep ? jw : 0.0f;
    }
    const float h = -0.5f * Lam;
    const float y0 = sA * y[0], y1 = sE * y[1], y2 = sT * y[2], y3 = sT * y[3], y4 = sA * y[4];
    const float i0 = y0 + y1 + y4;
    const float i1 = (vn - c) * y0 + vn * y1 + (vn + c) * y4;
    const float i2 = vt1 * i0 + y2;
    const float i3 = vt2 * i0 + y3;
    const float i4 = Hm * y0 + mid * y1 + vt1 * y2 + vt2 * y3 + Hp * y4;
    out[0] = h * i0;
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) out[1 + c3] = h * (en[c3] * i1 + et1[c3] * i2 + et2[c3] * i3);
    out[4] = h * i4;
}

struct Dir3FParams {
    Grid3 g;
    GasF gas;
    WenoF weno;
    int diss;
    const float* NF;          // float node fields [MF_COUNT][N]
    const float* NK;          // metrics of this direction [3][M] (float, from k3f_metric)
    const float* XD;          // the mesh velocity on the extended mesh [3][NE] (nullable: mesh at rest)
    float* RH;                // accumulated right-hand sides [6][N] (float)
    int first, last;
    int tma;                  // xi_2 / xi_3: node fields staged by TMA (persistent grid)
    int mode;
    float ca, cb, ca_lo, cb_lo;
    double dt_host;
    const double* dt_dev;
    const float *JUn, *Jn, *JUs, *Js;   // double-float planes
    float *JUo, *Jo;
    DevStatus* status;
};

template <int LB, int W>
struct PencilF {
    static constexpr int LS = (LB + 6) | 1;
    static constexpr int NB = W * LS;
    static constexpr int PL = 3 * LB + 6;
    static constexpr int NP = W * PL;
    static constexpr int NF = W * (LB + 1);
    static constexpr int NJ = W * (LB + 5);
    static constexpr size_t SMEM = sizeof(float) * (size_t(MS_COUNT) * NB + 5 * NP + 6 * NF + 5 * NJ);
    // TMA staging of the node fields of a xi_2 / xi_3 pencil: [MF_COUNT][LB + 6][W] floats, in 128-byte units
    static constexpr int STG = (W * (LB + 6) * MF_COUNT + 31) / 32 * 32;
    static constexpr size_t STG_BYTES = sizeof(float) * size_t(W) * (LB + 6) * MF_COUNT;
};

// ---------------------------------------------------------------- TMA staging
// The xi_2 and xi_3 kernels run persistent: a CTA takes pencils p, p + gridDim.x, ... and, while it
// computes one, the tensor-memory accelerator copies the next pencil's node fields (a box of W lines
// along xi_1 x (LB + 6) nodes along xi_k x all MF_COUNT field planes, one cp.async.bulk.tensor) into
// the staging buffer.  The box starts at xi_1 = a0, a multiple of W >= 4 floats (16 bytes), and the
// field planes have a row pitch of n1 floats, a multiple of 4 (checked when the map is built); the
// box may reach past the mesh along xi_k and xi_1, where the copy fills zeros: those nodes are the
// ghosts and the clamped lines, which the fill phase takes by plain loads or from the clamped line.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bounded wait for the phase of the given parity; false when it did not complete in 2^20 polls
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (int i = 0; i < (1 << 20); ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// one thread: the copy of pencil (a0, b, s0) into stg, completing on bar
template <int K, int LB>
__device__ __forceinline__ void stage_pencil(float* stg, const CUtensorMap* map, unsigned long long* bar,
                                             uint32_t bytes, int a0, int b, int s0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");    // the fill phase's reads of stg come first
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    const int c1 = K == 1 ? s0 - 3 : b, c2 = K == 1 ? b : s0 - 3;
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(stg)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(a0), "r"(c1), "r"(c2), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

template <int K, int LB, int W, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k3_dir_f(const __grid_constant__ Dir3FParams P,
                                                     const __grid_constant__ CUtensorMap tmap) {
    using PC = PencilF<LB, W>;
    constexpr int LS = PC::LS, NB = PC::NB, NP = PC::NP, NFc = PC::NF, NJ = PC::NJ;
    extern __shared__ __align__(128) float smf[];
    __shared__ __align__(8) unsigned long long bar;
    const bool tma = K != 0 && P.tma;
    float* STG = smf;
    float* S = smf + (tma ? PC::STG : 0);
    float* PB = S + MS_COUNT * NB;
    float* FB = PB + 5 * NP;
    float* JB = FB + 6 * NFc;
    const Grid3& g = P.g;
    const int tid = threadIdx.x;
    const int nk = g.n[K];
    const int nA = K == 0 ? g.n[1] : g.n[0];
    const int nB = K == 2 ? g.n[1] : g.n[2];
    const int nseg = (nk + LB - 1) / LB;
    const int ngA = (nA + W - 1) / W;
    const int total = nseg * ngA * nB;
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    const double dtd = P.dt_dev ? *P.dt_dev : P.dt_host;
    if (P.mode == 0 && P.dt_dev && dtd == 0.0) return;   // finished run
    const float dt = float(dtd);
    const int M1 = g.n[0] + (K == 0 ? 6 : 0), M2 = g.n[1] + (K == 1 ? 6 : 0), M3 = g.n[2] + (K == 2 ? 6 : 0);
    const size_t M = size_t(M1) * M2 * M3;
    const int M1e = g.n[0] + 6, M2e = g.n[1] + 6, M3e = g.n[2] + 6;     // the extended mesh (3 ghosts each way)
    const GasF& G = P.gas;
    const uint32_t stg_bytes = uint32_t(PC::STG_BYTES);
    if (tma) {
        if (tid == 0) {
            mbar_init(&bar);
            if (int(blockIdx.x) < total) {
                const int p = blockIdx.x, grp = p / nseg;
                stage_pencil<K, LB>(STG, &tmap, &bar, stg_bytes, (grp % ngA) * W, grp / ngA, (p % nseg) * LB);
            }
        }
        __syncthreads();
    }

    int iter = 0;
    for (int pen = blockIdx.x; pen < total; pen += tma ? int(gridDim.x) : total, ++iter) {   // plain: once
        const int seg = pen % nseg;
        const int grp = pen / nseg;
        const int a0 = (grp % ngA) * W;
        const int b = grp / ngA;
        const int s0 = seg * LB;
        if (tma) {
            // every thread waits for the copy itself (the acquire makes it visible); the CTA leaves together if
            // it did not arrive
            const bool ok = mbar_wait(&bar, uint32_t(iter & 1));
            if (!__syncthreads_and(ok)) {
                if (tid == 0) {
                    raise_error(P.status, ES_ERR_TIMEOUT, pen);
                    mbar_wait(&bar, uint32_t(iter & 1));         // the copy in flight, once more with the limit
                }
                return;
            }
        }

        // ---- A: node fields and metrics of the pencils
        for (int t = tid; t < W * (LB + 6); t += NT) {
            int line, q;
            if (K == 0) { line = t / (LB + 6); q = t % (LB + 6); }
            else { q = t / W; line = t % W; }
            int a = a0 + line;
            if (a > nA - 1) a = nA - 1;
            const int s = s0 + q - 3;
            const int ss = state_index(s, nk, g.bc[K]);
            int i1, i2, i3, j1, j2, j3;
            if (K == 0) { i1 = ss; i2 = a; i3 = b; }
            else if (K == 1) { i1 = a; i2 = ss; i3 = b; }
            else { i1 = a; i2 = b; i3 = ss; }
            const size_t id = idx3(g, i1, i2, i3);
            const int bx = line * LS + q;
            float v[MF_COUNT];                                   // all loads in flight before the stores
            if (tma && s >= 0 && s < nk) {                       // the staged copy: line a - a0 of the box
#pragma unroll
                for (int f = 0; f < MF_COUNT; ++f) v[f] = STG[(f * (LB + 6) + q) * W + (a - a0)];
            } else {
#pragma unroll
                for (int f = 0; f < MF_COUNT; ++f) v[f] = P.NF[f * N + id];
            }
#pragma unroll
            for (int f = 0; f < MF_COUNT; ++f) S[f * NB + bx] = v[f];
            int se = s + 3;
            se = se < 0 ? 0 : (se > nk + 5 ? nk + 5 : se);
            if (K == 0) { j1 = se; j2 = a; j3 = b; }
            else if (K == 1) { j1 = a; j2 = se; j3 = b; }
            else { j1 = a; j2 = b; j3 = se; }
            const size_t mi = (size_t(j3) * M2 + j2) * M1 + j1;
            const float nx = P.NK[mi], ny = P.NK[M + mi], nz = P.NK[2 * M + mi];
            S[M_NX * NB + bx] = nx;
            S[M_NY * NB + bx] = ny;
            S[M_NZ * NB + bx] = nz;
            float xt = 0.0f;
            if (P.XD) {     // J xi_{k,t} = -xdot . n_k, xdot from the extended mesh (its ghosts: the coordinates' rule)
                const size_t NE = size_t(M1e) * M2e * M3e;
                size_t e;
                if (K == 0) e = (size_t(b + 3) * M2e + (a + 3)) * M1e + se;
                else if (K == 1) e = (size_t(b + 3) * M2e + se) * M1e + (a + 3);
                else e = (size_t(se) * M2e + (b + 3)) * M1e + (a + 3);
                xt = -(P.XD[e] * nx + P.XD[NE + e] * ny + P.XD[2 * NE + e] * nz);
            }
            S[M_XT * NB + bx] = xt;
        }
        __syncthreads();
        if (tma && tid == 0 && pen + int(gridDim.x) < total) {    // the staging buffer is free: next pencil
            const int p = pen + gridDim.x, gp = p / nseg;
            stage_pencil<K, LB>(STG, &tmap, &bar, stg_bytes, (gp % ngA) * W, gp / ngA, (p % nseg) * LB);
        }

        // ---- C: pair fluxes, and B: neighbour jumps V_{q+1} - V_q, q = 0 .. LB+4 (eq. jumpV)
        for (int t = tid; t < NP; t += NT) {
            const int line = t / PC::PL, kk = t % PC::PL;
            int m, q;
            if (kk < LB + 1) { m = 1; q = 2 + kk; }
            else if (kk < 2 * LB + 3) { m = 2; q = 1 + (kk - LB - 1); }
            else { m = 3; q = kk - 2 * LB - 3; }
            const int l = line * LS + q, r = l + m;
            const float nx = 0.5f * (S[M_NX * NB + l] + S[M_NX * NB + r]);
            const float ny = 0.5f * (S[M_NY * NB + l] + S[M_NY * NB + r]);
            const float nz = 0.5f * (S[M_NZ * NB + l] + S[M_NZ * NB + r]);
            const float xt = 0.5f * (S[M_XT * NB + l] + S[M_XT * NB + r]);
            float f[5];
            pair_flux3_f(S, NB, l, r, nx, ny, nz, xt, G, f);
#pragma unroll
            for (int c = 0; c < 5; ++c) PB[c * NP + t] = f[c];
        }
        if (P.diss) {
            for (int t = tid; t < NJ; t += NT) {
                const int line = t / (LB + 5), q = t % (LB + 5);
                const int l = line * LS + q;
                float dV[5];
                entropy_jump3_f(S, NB, l, l + 1, G, dV);
#pragma unroll
                for (int c = 0; c < 5; ++c) JB[c * NJ + t] = dV[c];
            }
        }
        __syncthreads();

        // ---- D: face fluxes
        for (int t = tid; t < NFc; t += NT) {
            const int line = t / (LB + 1), f = t % (LB + 1);
            const int q = 2 + f;
            const int pbase = line * PC::PL;
            const int base = line * LS;
            float F[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            float FJ = 0.0f;
#pragma unroll
            for (int m = 1; m <= 3; ++m) {
                const int off = m == 1 ? 0 : (m == 2 ? LB + 1 : 2 * LB + 3);
                const float al = float(ec_alpha(m));
                for (int s = 0; s < m; ++s) {
                    const int qq = q - s;
                    const int pi = pbase + off + (qq - (3 - m));
#pragma unroll
                    for (int c = 0; c < 5; ++c) F[c] += al * PB[c * NP + pi];
                    FJ += al * 0.5f * (S[M_XT * NB + base + qq] + S[M_XT * NB + base + qq + m]);
                }
            }
            if (P.diss) {
                const int l = base + q;
                const float nx = 0.5f * (S[M_NX * NB + l] + S[M_NX * NB + l + 1]);
                const float ny = 0.5f * (S[M_NY * NB + l] + S[M_NY * NB + l + 1]);
                const float nz = 0.5f * (S[M_NZ * NB + l] + S[M_NZ * NB + l + 1]);
                const float xtf = 0.5f * (S[M_XT * NB + l] + S[M_XT * NB + l + 1]);
                float d[5];
                face_dissipation3_f(S, NB, l, nx, ny, nz, xtf, G, P.weno, d, P.status, JB, NJ, line * (LB + 5) + q);
#pragma unroll
                for (int c = 0; c < 5; ++c) F[c] += d[c];
            }
#pragma unroll
            for (int c = 0; c < 5; ++c) FB[c * NFc + t] = F[c];
            FB[5 * NFc + t] = FJ;
        }
        __syncthreads();

        // ---- E: divergence, accumulated in float; the last direction writes double-float results
        const float inv = g.finv[K];
        for (int t = tid; t < W * LB; t += NT) {
            int line, pos;
            if (K == 0) { line = t / LB; pos = t % LB; }
            else { pos = t / W; line = t % W; }
            const int a = a0 + line, s = s0 + pos;
            if (a >= nA || s >= nk) continue;
            int i1, i2, i3;
            if (K == 0) { i1 = s; i2 = a; i3 = b; }
            else if (K == 1) { i1 = a; i2 = s; i3 = b; }
            else { i1 = a; i2 = b; i3 = s; }
            const size_t id = idx3(g, i1, i2, i3);
            const int fm = line * (LB + 1) + pos;
            // every global operand of this node is loaded before the first global store (as far as the
            // compiler knows a store may alias a later load, which would serialise one round trip per component)
            float rh[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            float uh[6], ul[6], sh[6], sl[6];
            if (!P.first) {
#pragma unroll
                for (int c = 0; c < 6; ++c) rh[c] = P.RH[c * N + id];
            }
            const bool combine = P.last && P.mode != 1;
            if (combine) {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const float* un = c < 5 ? P.JUn + c * N : P.Jn;
                    const float* us = c < 5 ? P.JUs + c * N : P.Js;
                    const size_t lo = c < 5 ? 5 * N : N;
                    sh[c] = us[id];
                    sl[c] = us[lo + id];
                    uh[c] = P.ca != 0.0f ? un[id] : 0.0f;
                    ul[c] = P.ca != 0.0f ? un[lo + id] : 0.0f;
                }
            }
            float acc[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                acc[c] = -(FB[c * NFc + fm + 1] - FB[c * NFc + fm]) * inv;
                if (!P.first) acc[c] += rh[c];
            }
            if (!P.last) {
#pragma unroll
                for (int c = 0; c < 6; ++c) P.RH[c * N + id] = acc[c];
            } else if (P.mode == 1) {
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    P.JUo[c * N + id] = acc[c];
                    P.JUo[5 * N + c * N + id] = 0.0f;
                }
                P.Jo[id] = acc[5];
                P.Jo[N + id] = 0.0f;
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    float* uo = c < 5 ? P.JUo + c * N : P.Jo;
                    const size_t lo = c < 5 ? 5 * N : N;
                    const df Un = {uh[c], ul[c]};
                    const df Us = {sh[c], sl[c]};
                    const df inc = df_add_f(Us, dt * acc[c]);
                    df outv = df_mul(inc, {P.cb, P.cb_lo});
                    if (P.ca != 0.0f) outv = df_add(outv, df_mul(Un, {P.ca, P.ca_lo}));
                    uo[id] = outv.hi;
                    uo[lo + id] = outv.lo;
                    if (c == 5 && !(outv.hi > 0.0f)) raise_error(P.status, ES_ERR_MESH, int(id));
                }
            }
        }
        __syncthreads();                                      // S, PB, FB and JB are refilled next
    }
}

int g_nsm = 0;                 // SMs of the device (the persistent grids), set by d3f_prepare

template <int K, int LB, int W, int NT, int MINB>
static cudaError_t prep_shape() {
    const size_t smem = PencilF<LB, W>::SMEM + (K != 0 ? sizeof(float) * PencilF<LB, W>::STG : 0);
    return cudaFuncSetAttribute(k3_dir_f<K, LB, W, NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

template <int K, int LB, int W, int NT, int MINB>
static cudaError_t launch_shape(const Dir3FParams& P, const CUtensorMap& map, cudaStream_t s) {
    const Grid3& g = P.g;
    const int nA = K == 0 ? g.n[1] : g.n[0];
    const int nB = K == 2 ? g.n[1] : g.n[2];
    const long long blocks = (long long)((g.n[K] + LB - 1) / LB) * ((nA + W - 1) / W) * nB;
    const bool tma = K != 0 && P.tma;
    const long long resident = (long long)(g_nsm > 0 ? g_nsm : 1) * MINB;
    const long long grid = tma && blocks > resident ? resident : blocks;
    const size_t smem = PencilF<LB, W>::SMEM + (tma ? sizeof(float) * PencilF<LB, W>::STG : 0);
    k3_dir_f<K, LB, W, NT, MINB><<<unsigned(grid), NT, smem, s>>>(P, map);
    return cudaGetLastError();
}

// pencil shapes of the float kernels: 16 x 16 lines / 288 threads (two CTAs per SM), 32 x 8 / 288,
// 16 x 8 / 160 (three per SM), 32 x 4 / 160
template <int K>
static cudaError_t prep_dir() {
    cudaError_t e = prep_shape<K, 16, 16, 288, 2>();
    if (e == cudaSuccess) e = prep_shape<K, 32, 8, 288, 2>();
    if (e == cudaSuccess) e = prep_shape<K, 16, 8, 160, 3>();
    if (e == cudaSuccess) e = prep_shape<K, 32, 4, 160, 3>();
    return e;
}

template <int K>
static cudaError_t launch_dir(const Dir3FParams& P, const CUtensorMap& map, int shape, cudaStream_t s) {
    switch (shape) {
        case 1: return launch_shape<K, 32, 8, 288, 2>(P, map, s);
        case 2: return launch_shape<K, 16, 8, 160, 3>(P, map, s);
        case 3: return launch_shape<K, 32, 4, 160, 3>(P, map, s);
        default: return launch_shape<K, 16, 16, 288, 2>(P, map, s);
    }
}

// the driver's tensor-map encoder (fetched once; nullptr if the driver has none)
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// the tensor map of the float node fields [MF_COUNT][n3][n2][n1] with the box of one xi_k pencil (k = 1, 2):
// W nodes along xi_1, LB + 6 along xi_k, 1 along the third direction, all field planes.  Plain loads (false)
// when n1 is not a multiple of 4 (TMA strides are multiples of 16 bytes) or the encoder refuses.
template <int LB, int W>
static bool build_tmap(Ctx3* d, int k, int shape) {
    const Grid3& g = d->g;
    if (g.n[0] % 4 != 0) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    CUtensorMap m;
    const cuuint64_t dims[4] = {cuuint64_t(g.n[0]), cuuint64_t(g.n[1]), cuuint64_t(g.n[2]), cuuint64_t(MF_COUNT)};
    const cuuint64_t strides[3] = {cuuint64_t(g.n[0]) * 4, cuuint64_t(g.n[0]) * g.n[1] * 4, cuuint64_t(d->N) * 4};
    const cuuint32_t box[4] = {cuuint32_t(W), cuuint32_t(k == 1 ? LB + 6 : 1), cuuint32_t(k == 2 ? LB + 6 : 1),
                               cuuint32_t(MF_COUNT)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d->NF, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    static_assert(sizeof(CUtensorMap) == sizeof(d->tmap[0][0]), "tensor map size");
    memcpy(d->tmap[k - 1][shape], &m, sizeof(m));
    return true;
}

static bool tmap_for(Ctx3* d, int k, int shape, CUtensorMap* out) {
    if (k == 0 || d->no_tma) return false;
    int& st = d->tmap_state[k - 1][shape];
    if (st == 0) {
        bool ok;
        switch (shape) {
            case 1: ok = build_tmap<32, 8>(d, k, shape); break;
            case 2: ok = build_tmap<16, 8>(d, k, shape); break;
            case 3: ok = build_tmap<32, 4>(d, k, shape); break;
            default: ok = build_tmap<16, 16>(d, k, shape); break;
        }
        st = ok ? 1 : -1;
    }
    if (st != 1) return false;
    memcpy(out, d->tmap[k - 1][shape], sizeof(*out));
    return true;
}

// ---------------------------------------------------------------- metrics in double-float
// The cross-form metrics of eq. SCLCoeff formed as the FP64 path forms them (k3_coords, k3_deriv, k3_metric:
// stage coordinates on the mesh extended by 3 ghosts, the products delta_l[x_p] x_q once per node, and each
// direction's metric from differences of those products), in double-float arithmetic on the FP32 pipe: the
// stage coordinates are split into (hi, lo) floats once and every product and difference keeps a 48-bit
// significand, so the metric is rounded once, to the float the direction kernels read.  On GB300 the FP64
// version of these three kernels took more time than the float direction kernels.
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, {-b.hi, -b.lo}); }

// the coordinates of x_s = xn + cst dt xdot on the extended grid as (hi, lo) planes: XEh [3][NE], XEl [3][NE]
__global__ void k3f_coords(Grid3 g, const double* xn, const double* xdot, double cst, const double* dt_dev,
                           double dt_host, float* XEh, float* XEl) {
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    const unsigned E1 = g.n[0] + 6, E2 = g.n[1] + 6, E3 = g.n[2] + 6;
    const size_t NE = size_t(E1) * E2 * E3;
    const double cdt = cst * (dt_dev ? *dt_dev : dt_host);
    for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < NE; e += size_t(gridDim.x) * blockDim.x) {
        const unsigned eu = unsigned(e);                      // NE < 2^31 (es_create limits N to 2^30)
        const int i1 = int(eu % E1) - 3, i2 = int((eu / E1) % E2) - 3, i3 = int(eu / (E1 * E2)) - 3;
        const bool in = inside3(g, i1, i2, i3, 0);
        const size_t id = in ? idx3(g, i1, i2, i3) : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v;
            if (in) v = xdot ? xn[c * N + id] + cdt * xdot[c * N + id] : xn[c * N + id];
            else v = ghost_value3(g, xn + c * N, xdot ? xdot + c * N : nullptr, cdt, i1, i2, i3, c);
            float hi, lo;
            bits::split(v, hi, lo);                          // integer operations, not FP64 conversions
            XEh[c * NE + e] = hi;
            XEl[c * NE + e] = lo;
        }
    }
}

// the mesh velocity on the extended mesh as floats XD [3][NE]: the ghost rule of the coordinates without their
// period shift (a ghost's coordinate is the ghost rule's combination of x^n + c dt xdot plus the shift, so its
// velocity is the same combination of xdot)
__global__ void k3f_xdot_ext(Grid3 g, const double* xdot, float* XD) {
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    const unsigned E1 = g.n[0] + 6, E2 = g.n[1] + 6, E3 = g.n[2] + 6;
    const size_t NE = size_t(E1) * E2 * E3;
    for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < NE; e += size_t(gridDim.x) * blockDim.x) {
        const unsigned eu = unsigned(e);
        const int i1 = int(eu % E1) - 3, i2 = int((eu / E1) % E2) - 3, i3 = int(eu / (E1 * E2)) - 3;
        const bool in = inside3(g, i1, i2, i3, 0);
        const size_t id = in ? idx3(g, i1, i2, i3) : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            XD[c * NE + e] = float(in ? xdot[c * N + id] : ghost_value3(g, xdot + c * N, nullptr, 0.0, i1, i2, i3, -1));
    }
}

// XE += f dt XD in double-float (f = the change of the stage-time fraction; dt from the device or the host)
__global__ void k3f_coords_add(size_t NE, float* XEh, float* XEl, const float* XD, double f, const double* dt_dev,
                               double dt_host) {
    const float a = float(f * (dt_dev ? *dt_dev : dt_host));
    for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < 3 * NE; e += size_t(gridDim.x) * blockDim.x) {
        const df v = df_add_f({XEh[e], XEl[e]}, a * XD[e]);
        XEh[e] = v.hi;
        XEl[e] = v.lo;
    }
}

// D[3 l + j] = delta_l[x_p] x_q (p = (j + 1) % 3, q = (j + 2) % 3; delta_l undivided, 0 where the xi_l index is
// not interior) as (hi, lo) planes Dh, Dl [9][NE]
__global__ void k3f_deriv(Grid3 g, const float* XEh, const float* XEl, float* Dh, float* Dl) {
    const unsigned E1 = g.n[0] + 6, E2 = g.n[1] + 6, E3 = g.n[2] + 6;
    const size_t NE = size_t(E1) * E2 * E3;
    const size_t st[3] = {1, size_t(E1), size_t(E1) * E2};
    for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < NE; e += size_t(gridDim.x) * blockDim.x) {
        const unsigned eu = unsigned(e);
        const int ee[3] = {int(eu % E1), int((eu / E1) % E2), int(eu / (E1 * E2))};
        const df x[3] = {{XEh[e], XEl[e]}, {XEh[NE + e], XEl[NE + e]}, {XEh[2 * NE + e], XEl[2 * NE + e]}};
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const bool ok = ee[l] >= 3 && ee[l] < g.n[l] + 3;
            df dl[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                df acc = {0.0f, 0.0f};
                if (ok) {
#pragma unroll
                    for (int m = 1; m <= 3; ++m) {
                        const size_t up = p * NE + e + m * st[l], dn = p * NE + e - m * st[l];
                        const df d = df_sub({XEh[up], XEl[up]}, {XEh[dn], XEl[dn]});
                        acc = df_add(acc, df_mul_f(d, float(0.5 * ec_alpha(m))));
                    }
                }
                dl[p] = acc;
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const df v = df_mul(dl[(j + 1) % 3], x[(j + 2) % 3]);
                Dh[(3 * l + j) * NE + e] = v.hi;
                Dl[(3 * l + j) * NE + e] = v.lo;
            }
        }
    }
}

// J dxi_k/dx_j on direction k's grid (n_k + 6 nodes along xi_k, interior across), rounded to float [3][M]
// (the direction is a template parameter: no run-time indexing of the grid's arrays)
template <int k>
__global__ void k3f_metric(Grid3 g, const float* Dh, const float* Dl, float* NKo) {
    const unsigned E1 = g.n[0] + 6, E2 = g.n[1] + 6;
    const size_t NE = size_t(E1) * E2 * (g.n[2] + 6);
    unsigned m1 = g.n[0], m2 = g.n[1], m3 = g.n[2];
    if (k == 0) m1 += 6;
    else if (k == 1) m2 += 6;
    else m3 += 6;
    const size_t M = size_t(m1) * m2 * m3;
    const int l = (k + 1) % 3, m = (k + 2) % 3;
    const float scale = float(g.inv_dxi[l] * g.inv_dxi[m]);
    const size_t stl = l == 0 ? 1 : (l == 1 ? size_t(E1) : size_t(E1) * E2);
    const size_t stm = m == 0 ? 1 : (m == 1 ? size_t(E1) : size_t(E1) * E2);
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < M; t += size_t(gridDim.x) * blockDim.x) {
        const unsigned tu = unsigned(t);
        const int a1 = int(tu % m1), a2 = int((tu / m1) % m2), a3 = int(tu / (m1 * m2));
        const size_t e = eidx(g, a1 + (k == 0 ? 0 : 3), a2 + (k == 1 ? 0 : 3), a3 + (k == 2 ? 0 : 3));
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const size_t ol = size_t(3 * l + j) * NE, om = size_t(3 * m + j) * NE;    // delta_l[x_p] x_q, delta_m[...]
            df A = {0.0f, 0.0f}, B = {0.0f, 0.0f};
#pragma unroll
            for (int a = 1; a <= 3; ++a) {
                const float h = float(0.5 * ec_alpha(a));
                const size_t sm = a * stm, sl = a * stl;
                A = df_add(A, df_mul_f(df_sub({Dh[ol + e + sm], Dl[ol + e + sm]}, {Dh[ol + e - sm], Dl[ol + e - sm]}), h));
                B = df_add(B, df_mul_f(df_sub({Dh[om + e + sl], Dl[om + e + sl]}, {Dh[om + e - sl], Dl[om + e - sl]}), h));
            }
            const df diff = df_sub(A, B);
            NKo[j * M + t] = (diff.hi + diff.lo) * scale;
        }
    }
}

// CFL (eq. cfl) from the float node fields and the FP64 metrics: J xi_{k,t} = -xdot . n_k, xdot = nullptr
// is a mesh at rest; the maximum goes to d->red[slot]
__global__ void k3_cfl_f(Grid3 g, Gas Gd, const float* NF, const float* J, const float* NK0, const float* NK1,
                         const float* NK2, const double* xdot, int slot, DevScalars* d) {
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    const size_t M[3] = {size_t(g.n[0] + 6) * g.n[1] * g.n[2], size_t(g.n[0]) * (g.n[1] + 6) * g.n[2],
                         size_t(g.n[0]) * g.n[1] * (g.n[2] + 6)};
    const float* NK[3] = {NK0, NK1, NK2};
    const float a = float(Gd.a), R = float(Gd.R), delta = float(Gd.delta);
    float mx = 0.0f;
    for (size_t id = blockIdx.x * size_t(blockDim.x) + threadIdx.x; id < N; id += size_t(gridDim.x) * blockDim.x) {
        const int i1 = int(id % g.n[0]), i2 = int((id / g.n[0]) % g.n[1]), i3 = int(id / (size_t(g.n[0]) * g.n[1]));
        const float rho = NF[M_RHO * N + id], T = NF[M_T * N + id], iom = NF[M_IOM * N + id];
        const float v[3] = {NF[M_V1 * N + id], NF[M_V2 * N + id], NF[M_V3 * N + id]};
        const float c2 = (1.0f + delta) * R * T * (iom * iom) - 2.0f * a * rho;
        const float c = sqrtf(fmaxf(c2, 0.0f));
        const float iJ = 1.0f / J[id];
        const float vr[3] = {v[0] - (xdot ? float(xdot[id]) : 0.0f), v[1] - (xdot ? float(xdot[N + id]) : 0.0f),
                             v[2] - (xdot ? float(xdot[2 * N + id]) : 0.0f)};      // velocity relative to the mesh
        float tot = 0.0f;
        for (int k = 0; k < 3; ++k) {
            const int m1 = g.n[0] + (k == 0 ? 6 : 0), m2 = g.n[1] + (k == 1 ? 6 : 0);
            const size_t mi = (size_t(i3 + (k == 2 ? 3 : 0)) * m2 + i2 + (k == 1 ? 3 : 0)) * m1 + i1 + (k == 0 ? 3 : 0);
            const float n0 = NK[k][mi], n1 = NK[k][M[k] + mi], n2 = NK[k][2 * M[k] + mi];
            tot += (fabsf(n0 * vr[0] + n1 * vr[1] + n2 * vr[2]) + sqrtf(n0 * n0 + n1 * n1 + n2 * n2) * c) * iJ *
                   g.finv[k];
        }
        if (!(c2 > 0.0f)) tot = 3.0e38f;
        mx = fmaxf(mx, tot);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomic_max_pos(&d->red[slot], double(mx));
}

// J (FP64, from the FP64 kernel) into double-float planes
__global__ void k3_split(const double* a, float* out, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const float hi = float(a[i]);
        out[i] = hi;
        out[n + i] = float(a[i] - double(hi));
    }
}


// ---------------------------------------------------------------- mesh redistribution (Sec. 4)
// On the FP32 pipe, with the Jacobi iteration written for the displacement delta = x - x^n from
// the mesh at t^n.  omega is fixed during the sweeps, so x^[nu+1]_i = sum_nb a_nb x^[nu]_nb with
// a_nb = w_nb / sum_nb w_nb becomes delta^[nu+1]_i = g_i + sum_nb a_nb delta^[nu]_nb, where
// g_i = sum_nb a_nb (x^n_nb - x^n_i) is formed once per solve in double-float from x^n on the
// extended mesh (the stage metrics' coordinates, ghosts with the period shift) and then rounded:
// the sweeps round only the displacement, which is small against the spacing.
// The mixed form has periodic and outflow ends only; every node on an outflow end is fixed, so a
// node that moves has its six neighbours in the mesh or across a periodic end, where delta wraps
// (x shifts by the period, delta does not).

__device__ __forceinline__ void split3(const Grid3& g, int id, int* ii) {
    const int r = id / g.n[0];
    ii[0] = id - r * g.n[0];
    ii[2] = r / g.n[1];
    ii[1] = r - ii[2] * g.n[1];
}

__device__ __forceinline__ int stride3i(const Grid3& g, int k) {
    return k == 0 ? 1 : (k == 1 ? g.n[0] : g.n[0] * g.n[1]);
}

// neighbour at s = +-1 along k, ghosts by copy (outflow) or wrap (periodic)
__device__ __forceinline__ int nb3(const Grid3& g, int id, int ik, int k, int s) {
    const int j = state_index(ik + s, g.n[k], g.bc[k]);
    return id + (j - ik) * stride3i(g, k);
}

__device__ __forceinline__ bool fixed_node3(const Grid3& g, const int* ii) {
    bool f = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) f = f || (g.bc[k] != ES_BC_PERIODIC && (ii[k] == 0 || ii[k] == g.n[k] - 1));
    return f;
}

__device__ __forceinline__ float warp_max_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_min_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// the raw monitor terms of eq. van der Waalsmonitor (or the smooth-test monitor) from the
// float density and G: central first and second differences along each direction
// rhoF, GF: (hi, lo) float planes of the density and G (k_mon_fields_f); the differences of neighbours
// are taken in double-float arithmetic and then rounded
__global__ void k3f_mon_terms(Grid3 g, MonitorParams mp, const float* rhoF, const float* GF, float* t0, float* t1,
                              float* t2, DevScalars* d) {
    const int N = g.n[0] * g.n[1] * g.n[2];
    float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        int ii[3];
        split3(g, id, ii);
        const df r0 = {rhoF[id], rhoF[N + id]}, G0 = {GF[id], GF[N + id]};
        float gr = 0.0f, gg = 0.0f, lg = 0.0f, lr = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float h = g.finv[k];
            const int ip = nb3(g, id, ii[k], k, 1), im = nb3(g, id, ii[k], k, -1);
            const df rp = {rhoF[ip], rhoF[N + ip]}, rm = {rhoF[im], rhoF[N + im]};
            const df Gp = {GF[ip], GF[N + ip]}, Gm = {GF[im], GF[N + im]};
            const float a = df_diff(rp, rm) * 0.5f * h, b = df_diff(Gp, Gm) * 0.5f * h;
            const float c = df_second_diff(Gp, G0, Gm) * h * h, e = df_second_diff(rp, r0, rm) * h * h;
            gr += a * a;
            gg += b * b;
            lg += c * c;
            lr += e * e;
        }
        float v0, v1, v2;
        if (mp.kind == ES_MONITOR_SMOOTH) {
            v0 = sqrtf(gr);
            v1 = 0.0f;
            v2 = sqrtf(lr);
        } else {
            v0 = gr;
            v1 = mp.kappa >= 2 ? gg : 0.0f;
            v2 = lg;
        }
        t0[id] = v0;
        t1[id] = v1;
        t2[id] = v2;
        m0 = fmaxf(m0, v0);
        m1 = fmaxf(m1, v1);
        m2 = fmaxf(m2, v2);
    }
    m0 = warp_max_f(m0);
    m1 = warp_max_f(m1);
    m2 = warp_max_f(m2);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(&d->red[RED_MON0], double(m0));
        atomic_max_pos(&d->red[RED_MON1], double(m1));
        atomic_max_pos(&d->red[RED_MON2], double(m2));
    }
}

// omega_i <- sum_{j in {0,+-1}^3} (1/2)^(|j|_1 + 3) omega_{i+j} (Sec. 4's low-pass filter)
__global__ void k3f_filter(Grid3 g, const float* in, float* out) {
    const int N = g.n[0] * g.n[1] * g.n[2];
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        int ii[3];
        split3(g, id, ii);
        int o1[3], o2[3], o3[3];
        o1[1] = o2[1] = o3[1] = 0;
        o1[0] = nb3(g, id, ii[0], 0, -1) - id;
        o1[2] = nb3(g, id, ii[0], 0, 1) - id;
        o2[0] = nb3(g, id, ii[1], 1, -1) - id;
        o2[2] = nb3(g, id, ii[1], 1, 1) - id;
        o3[0] = nb3(g, id, ii[2], 2, -1) - id;
        o3[2] = nb3(g, id, ii[2], 2, 1) - id;
        float s = 0.0f;
#pragma unroll
        for (int d3 = 0; d3 < 3; ++d3) {
            float pl = 0.0f;
#pragma unroll
            for (int d2 = 0; d2 < 3; ++d2) {
                const int b = id + o2[d2] + o3[d3];
                const float row = 0.25f * in[b + o1[0]] + 0.5f * in[b] + 0.25f * in[b + o1[2]];
                pl += (d2 == 1 ? 0.5f : 0.25f) * row;
            }
            s += (d3 == 1 ? 0.5f : 0.25f) * pl;
        }
        out[id] = s;
    }
}

// the sweep coefficients of every node: a_nb for the six neighbours ([6][N], order -xi_1, +xi_1,
// -xi_2, ...) and g ([3][N]); zero at fixed nodes
__global__ void k3f_coeffs(Grid3 g, const float* om, const float* XEh, const float* XEl, float* A, float* Gc) {
    const int N = g.n[0] * g.n[1] * g.n[2];
    const size_t P = size_t(N);
    const size_t NE = size_t(g.n[0] + 6) * (g.n[1] + 6) * (g.n[2] + 6);
    const size_t est[3] = {1, size_t(g.n[0] + 6), size_t(g.n[0] + 6) * (g.n[1] + 6)};
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        int ii[3];
        split3(g, id, ii);
        if (fixed_node3(g, ii)) {
#pragma unroll
            for (int m = 0; m < 6; ++m) A[m * P + id] = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) Gc[c * P + id] = 0.0f;
            continue;
        }
        const float w0 = om[id];
        float w[6], den = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float ih2 = g.finv2[k];
            w[2 * k] = 0.5f * (w0 + om[nb3(g, id, ii[k], k, -1)]) * ih2;
            w[2 * k + 1] = 0.5f * (w0 + om[nb3(g, id, ii[k], k, 1)]) * ih2;
            den += w[2 * k] + w[2 * k + 1];
        }
        const float iden = 1.0f / den;
        // x^n_nb - x^n_i from the extended mesh (ghosts with the period shift), in double-float
        const size_t e = eidx(g, ii[0] + 3, ii[1] + 3, ii[2] + 3);
        df gs[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float am = w[2 * k] * iden, ap = w[2 * k + 1] * iden;
            A[(2 * k) * P + id] = am;
            A[(2 * k + 1) * P + id] = ap;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t o = c * NE + e;
                const df xi = {XEh[o], XEl[o]};
                const df dm = df_sub({XEh[o - est[k]], XEl[o - est[k]]}, xi);
                const df dp = df_sub({XEh[o + est[k]], XEl[o + est[k]]}, xi);
                gs[c] = df_add(gs[c], df_add(df_mul_f(dm, am), df_mul_f(dp, ap)));
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) Gc[c * P + id] = gs[c].hi + gs[c].lo;
    }
}

// Jacobi sweep k on the displacement (sweep 0 starts from delta = 0 and writes da; sweep k reads
// buf[(k - 1) % 2] and writes buf[k % 2]); with `check` the last block to finish compares the
// grid's max change with eps and latches convergence, after which the remaining sweeps return
__global__ void k3f_jacobi(Grid3 g, const float* A, const float* Gc, float* da, float* db, int k, DevScalars* d,
                           int check, double eps) {
    if (d->conv) return;
    const int N = g.n[0] * g.n[1] * g.n[2];
    const size_t P = size_t(N);
    const float* din = k == 0 ? nullptr : (((k - 1) & 1) ? db : da);
    float* dout = (k & 1) ? db : da;
    float chg = 0.0f;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        int ii[3];
        split3(g, id, ii);
        if (fixed_node3(g, ii)) {
#pragma unroll
            for (int c = 0; c < 3; ++c) dout[c * P + id] = 0.0f;
            continue;
        }
        float v[3] = {Gc[id], Gc[P + id], Gc[2 * P + id]};
        if (din) {
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                const float am = A[(2 * kk) * P + id], ap = A[(2 * kk + 1) * P + id];
                const int im = nb3(g, id, ii[kk], kk, -1), ip = nb3(g, id, ii[kk], kk, 1);
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] += am * din[c * P + im] + ap * din[c * P + ip];
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            chg = fmaxf(chg, fabsf(v[c] - (din ? din[c * P + id] : 0.0f)));
            dout[c * P + id] = v[c];
        }
    }
    if (check) {
        chg = warp_max_f(chg);
        __shared__ float sh[32];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) sh[w] = chg;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.0f;
            for (int i = 0; i < int(blockDim.x + 31) / 32; ++i) m = fmaxf(m, sh[i]);
            atomic_max_pos(&d->red[RED_JAC], double(m));
            __threadfence();
            const unsigned int ticket = atomicAdd(&d->done, 1u);
            if (ticket == gridDim.x - 1) {
                const double c = __longlong_as_double((long long)atomicAdd(&d->red[RED_JAC], 0ULL));
                if (c < eps) d->conv = 1;
                d->red[RED_JAC] = 0ULL;
                d->done = 0u;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&d->sweeps, 1);
}

__device__ __forceinline__ const float* sweep_result(const DevScalars* d, const float* da, const float* db) {
    if (d->sweeps == 0) return nullptr;
    return ((d->sweeps - 1) & 1) ? db : da;
}

// Delta_gamma over all nodes and directions (Sec. 4): the spacing to the neighbour the node
// moves towards, over twice its displacement along that direction
__global__ void k3f_limiter(Grid3 g, const float* XEh, const float* XEl, const float* da, const float* db,
                            DevScalars* d) {
    const int N = g.n[0] * g.n[1] * g.n[2];
    const size_t P = size_t(N);
    const size_t NE = size_t(g.n[0] + 6) * (g.n[1] + 6) * (g.n[2] + 6);
    const size_t est[3] = {1, size_t(g.n[0] + 6), size_t(g.n[0] + 6) * (g.n[1] + 6)};
    const float* dl = sweep_result(d, da, db);
    float m = 1.0f;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; dl && id < N; id += gridDim.x * blockDim.x) {
        int ii[3];
        split3(g, id, ii);
        if (fixed_node3(g, ii)) continue;
        const size_t e = eidx(g, ii[0] + 3, ii[1] + 3, ii[2] + 3);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float dx = dl[k * P + id];
            const size_t o = k * NE + e;                       // component k of x^n along direction k
            if (dx < 0.0f)
                m = fminf(m, df_diff({XEh[o], XEl[o]}, {XEh[o - est[k]], XEl[o - est[k]]}) / (-2.0f * dx));
            else if (dx > 0.0f)
                m = fminf(m, df_diff({XEh[o + est[k]], XEl[o + est[k]]}, {XEh[o], XEl[o]}) / (2.0f * dx));
        }
    }
    m = warp_min_f(m);
    if ((threadIdx.x & 31) == 0) atomic_min_pos(&d->red[RED_GAMMA], double(m));
}

// xdot = Delta_gamma delta^[mu] / dt (FP64, the API's array)
__global__ void k3f_velocity(Grid3 g, const float* da, const float* db, DevScalars* d, double* xdot) {
    const int N = g.n[0] * g.n[1] * g.n[2];
    const size_t P = size_t(N);
    const float* dl = sweep_result(d, da, db);
    // Delta_gamma / dt once per block (an FP64 division); the velocity in float, widened from its bits
    __shared__ float fs;
    if (threadIdx.x == 0) {
        const double gam = __longlong_as_double((long long)d->red[RED_GAMMA]);
        const double dt = d->dt;
        fs = dt > 0.0 ? float(gam / dt) : 0.0f;
    }
    __syncthreads();
    const float f = fs;
    for (size_t id = blockIdx.x * size_t(blockDim.x) + threadIdx.x; id < 3 * P; id += size_t(gridDim.x) * blockDim.x)
        xdot[id] = dl ? bits::widen(f * dl[id]) : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d->gamma = __longlong_as_double((long long)d->red[RED_GAMMA]);
        d->sweeps_total += d->sweeps;
        d->solves += 1;
    }
}

}  // namespace mixed3

using namespace mixed3;

cudaError_t d3f_prepare() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = prep_dir<0>();
    if (e == cudaSuccess) e = prep_dir<1>();
    if (e == cudaSuccess) e = prep_dir<2>();
    return e;
}

static GasF gasf(const Gas& g) {
    GasF G;
    G.a = float(g.a);
    G.b = float(g.b);
    G.R = float(g.R);
    G.cv = float(g.cv);
    G.delta = float(g.delta);
    G.Rb = float(g.R * g.b);
    G.icv = float(1.0 / g.cv);
    G.iR = float(1.0 / g.R);
    G.idelta = float(g.cv / g.R);
    return G;
}

static WenoF wenof(const Weno& w) {
    WenoF W;
    W.g1 = float(w.g1);
    W.g2 = float(w.g2);
    W.g3 = float(w.g3);
    W.g12 = float(w.g12);
    W.ig22 = float(w.ig22);
    W.ig3 = float(w.ig3);
    W.eps = float(w.eps);
    W.sign_tol = float(w.sign_tol);
    return W;
}

int d3f_metrics(Ctx3* d, const double* xn, const double* xdot, double cst, const double* dt_dev, double dt_host,
                cudaStream_t s, const Stage3* inc) {
    const int G = d->grid;
    const size_t NE = d->NE;
    float* XEh = (float*)d->XE;                   // [3][NE] doubles hold the (hi, lo) float planes
    float* Dh = (float*)d->D;                     // [9][NE] likewise
    int n = 4;
    if (inc && xdot) {                            // within a step: move the coordinates the buffer holds (d->XD
                                                  // holds xdot: d3_stage formed it)
        k3f_coords_add<<<G, 256, 0, s>>>(NE, XEh, XEh + 3 * NE, d->XD, cst - inc->xe_cst, dt_dev, dt_host);
    } else {
        k3f_coords<<<G, 256, 0, s>>>(d->g, xn, cst != 0.0 ? xdot : nullptr, cst, dt_dev, dt_host, XEh, XEh + 3 * NE);
    }
    k3f_deriv<<<G, 256, 0, s>>>(d->g, XEh, XEh + 3 * NE, Dh, Dh + 9 * NE);
    k3f_metric<0><<<G, 256, 0, s>>>(d->g, Dh, Dh + 9 * NE, (float*)d->NK[0]);
    k3f_metric<1><<<G, 256, 0, s>>>(d->g, Dh, Dh + 9 * NE, (float*)d->NK[1]);
    k3f_metric<2><<<G, 256, 0, s>>>(d->g, Dh, Dh + 9 * NE, (float*)d->NK[2]);
    return n + 1;
}

int d3f_form_xd(Ctx3* d, const double* xdot, cudaStream_t s) {
    k3f_xdot_ext<<<d->grid, 256, 0, s>>>(d->g, xdot, d->XD);
    return 1;
}

int d3f_nodes(Ctx3* d, const void* JU, const void* J, DevStatus* st, cudaStream_t s) {
    k3_nodes_f<<<d->grid, 256, 0, s>>>(d->g, gasf(d->gas), (const float*)JU, (const float*)J, (float*)d->NF, st);
    return 1;
}

int d3f_cfl(Ctx3* d, const void* J, const double* xdot, int slot, DevScalars* dv, cudaStream_t s) {
    k3_cfl_f<<<d->grid, 256, 0, s>>>(d->g, d->gas, (const float*)d->NF, (const float*)J, (const float*)d->NK[0],
                                      (const float*)d->NK[1], (const float*)d->NK[2], xdot, slot, dv);
    return 1;
}

int d3f_init_J(Ctx3* d, const double* Jd, void* J, cudaStream_t s) {
    k3_split<<<d->grid, 256, 0, s>>>(Jd, (float*)J, d->N);
    return 1;
}

int d3f_directions(Ctx3* d, const Stage3& a, DevStatus* st, cudaStream_t s, cudaError_t* err) {
    Dir3FParams P;
    P.g = d->g;
    P.gas = gasf(d->gas);
    P.weno = wenof(d->weno);
    P.diss = d->diss;
    P.NF = (const float*)d->NF;
    P.XD = a.xdot ? d->XD : nullptr;          // d3_stage formed it from a.xdot
    P.RH = (float*)d->RH;
    P.mode = a.mode;
    P.ca = float(a.ca);
    P.cb = float(a.cb);
    P.ca_lo = float(a.ca - double(P.ca));
    P.cb_lo = float(a.cb - double(P.cb));
    P.dt_host = a.dt_host;
    P.dt_dev = a.dt_dev;
    P.JUn = (const float*)a.JUn;
    P.Jn = (const float*)a.Jn;
    P.JUs = (const float*)a.JUs;
    P.Js = (const float*)a.Js;
    P.JUo = (float*)a.JUo;
    P.Jo = (float*)a.Jo;
    P.status = st;
    cudaError_t e = cudaGetLastError();
    int n = 0;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        P.NK = (const float*)d->NK[k];
        P.first = k == 0;
        P.last = k == 2;
        CUtensorMap map;
        memset(&map, 0, sizeof(map));
        P.tma = tmap_for(d, k, d->shape, &map) ? 1 : 0;
        e = k == 0 ? launch_dir<0>(P, map, d->shape, s)
                   : (k == 1 ? launch_dir<1>(P, map, d->shape, s) : launch_dir<2>(P, map, d->shape, s));
        ++n;
    }
    *err = e;
    return e == cudaSuccess ? n : -1;
}

int d3f_mesh(Ctx3* d, const void* JU, const void* J, const double* xn, double* xdot, DevScalars* dv,
             cudaStream_t s, cudaError_t* err, bool xe_current) {
    const int G = d->grid;
    int n = 0;
    // the sweep coefficients and the limiter read x^n on the extended mesh as double-float planes, which the
    // step's time-step pass has just formed for its metrics (xe_current); otherwise form them here
    float* XEh = (float*)d->XE;
    float* XEl = XEh + 3 * d->NE;
    if (!xe_current) {
        k3f_coords<<<G, 256, 0, s>>>(d->g, xn, nullptr, 0.0, nullptr, 0.0, XEh, XEl);
        ++n;
    }
    // the elementwise kernels of the 1D/2D mixed path see the 3D mesh as N nodes in a row
    GridParams flat;
    flat.dim = 3;
    flat.n1 = int(d->N);
    flat.n2 = 1;
    flat.bc[0] = flat.bc[1] = ES_BC_PERIODIC;
    flat.inv_dxi[0] = flat.inv_dxi[1] = 1.0;
    flat.period[0] = flat.period[1] = 0.0;
    grid_floats(flat);
    float* rho = (float*)d->rhoF;
    float* Gf = (float*)d->GF;
    float* t0 = (float*)d->t0;
    float* t1 = (float*)d->t1;
    float* t2 = (float*)d->t2;
    float* om = (float*)d->om0;
    float* other = (float*)d->om1;
    float* A = (float*)d->xa;                     // [6][N] floats in the [3][N] doubles
    float* da = (float*)d->xb;                    // two [3][N] float displacements
    float* db = da + 3 * d->N;               // (xb holds [3][N] doubles)
    k_mon_fields_f<<<G, 256, 0, s>>>(flat, gas_f32(d->gas), (const float*)JU, (const float*)J, rho, Gf);
    k3f_mon_terms<<<G, 256, 0, s>>>(d->g, d->mon, rho, Gf, t0, t1, t2, dv);
    k_mon_omega_f<<<G, 256, 0, s>>>(flat, d->mon, t0, t1, t2, dv, om);
    n += 3;
    for (int k = 0; k < d->filter_passes; ++k) {
        k3f_filter<<<G, 256, 0, s>>>(d->g, om, other);
        ++n;
        float* t = om;
        om = other;
        other = t;
    }
    k3f_coeffs<<<G, 256, 0, s>>>(d->g, om, XEh, XEl, A, d->gc);
    ++n;
    const int check = d->eps > 0.0;
    for (int k = 0; k < d->sweeps; ++k) {
        k3f_jacobi<<<G, 256, 0, s>>>(d->g, A, d->gc, da, db, k, dv, check, d->eps);
        ++n;
    }
    k3f_limiter<<<G, 256, 0, s>>>(d->g, XEh, XEl, da, db, dv);
    k3f_velocity<<<G, 256, 0, s>>>(d->g, da, db, dv, xdot);
    n += 2;
    *err = cudaGetLastError();
    return *err == cudaSuccess ? n : -1;
}

}  // namespace es
