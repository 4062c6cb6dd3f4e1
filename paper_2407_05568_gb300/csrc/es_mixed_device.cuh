// es_mixed_device.cuh -- device functions of the mixed-precision form (FP32 pipe,
// double-float state and primitive jumps), shared by the tiled stage kernel and
// the batched persistent kernel.  See es_stage_mixed.cu for the design.
#pragma once
#include <cuda_runtime.h>

#include "es_device.cuh"
#include "es_df.cuh"
#include "es_internal.h"

namespace es {
namespace mixed {

enum FieldF {
    G_RHO, G_V1, G_V2, G_T, G_IT, G_OM, G_IOM, G_G, G_RT, G_VT1, G_VT2, G_V2T, G_RV1, G_RV2, G_RP,
    G_RHOL, G_V1L, G_V2L, G_TL,   // low parts of rho, v, T (double-float)
    G_N1X, G_N1Y, G_XT1, G_N2X, G_N2Y, G_XT2,
    G_COUNT
};

template <int DIM, int BX, int BY, int NT>
struct TileF {
    static constexpr int GX = BX + 6;
    static constexpr int GY = DIM == 2 ? BY + 6 : 1;
    static constexpr int NB = GX * GY;
    static constexpr int NC = DIM + 2;
    static constexpr int NP1 = (DIM == 2 ? BY : 1) * (3 * BX + 6);
    static constexpr int NP2 = DIM == 2 ? BX * (3 * BY + 6) : 0;
    static constexpr int NP = NP1 > NP2 ? NP1 : NP2;
    static constexpr int NF1 = (DIM == 2 ? BY : 1) * (BX + 1);
    static constexpr int NF2 = DIM == 2 ? BX * (BY + 1) : 0;
    static constexpr int NF = NF1 > NF2 ? NF1 : NF2;
    static constexpr int PAIR_FLOATS = (NP * NC > 4 * NB) ? NP * NC : 4 * NB;
    // entropy-variable jumps between neighbours along each line (box positions q, q + 1), shared
    // by the faces whose stencils contain them
    static constexpr int NJ1 = (DIM == 2 ? BY : 1) * (BX + 5);
    static constexpr int NJ2 = DIM == 2 ? BX * (BY + 5) : 0;
    static constexpr int NJ = NJ1 > NJ2 ? NJ1 : NJ2;
    static constexpr size_t SMEM =
        sizeof(float) * (size_t(G_COUNT) * NB + PAIR_FLOATS + NF * (NC + 1) + size_t(NJ) * NC);
    static_assert(NT >= BX * (DIM == 2 ? BY : 1) && NT % 32 == 0, "threads cover the tile");
};

struct GasF {
    float a, b, R, cv, delta, Rb, icv, iR, idelta;
};

struct WenoF {
    float g1, g2, g3, g12, ig22, ig3, eps, sign_tol;
};

// reciprocal logarithmic mean 1/{a}^ln from the relative jump f = (a_l - a_r)/(a_l + a_r):
// [[ln a]] = ln((1 + f)/(1 - f)) = 2 artanh(f); series of artanh(f)/f for |f| < 0.05
__device__ __forceinline__ float inv_log_mean_j(float al, float ar, float d) {
    // d = a_l - a_r, passed in when known to more digits than al - ar
    const float s = al + ar;
    const float is = 1.0f / s;
    const float f = d * is;
    if (fabsf(f) < 0.05f) {
        const float u = f * f;
        const float F = 1.0f + u * (1.0f / 3.0f + u * (1.0f / 5.0f + u * (1.0f / 7.0f + u * (1.0f / 9.0f))));
        return 2.0f * F * is;
    }
    return log1pf(2.0f * f / (1.0f - f)) / d;
}

__device__ __forceinline__ float inv_log_mean_f(float al, float ar) { return inv_log_mean_j(al, ar, al - ar); }

__device__ __forceinline__ float mr_weno5_f(float wm2, float wm1, float w0, float wp1, float wp2, const WenoF& c) {
    const float q2 = (-wm1 + 5.0f * w0 + 2.0f * wp1) * (1.0f / 6.0f);
    const float q3 = (2.0f * wm2 - 13.0f * wm1 + 47.0f * w0 + 27.0f * wp1 - 3.0f * wp2) * (1.0f / 60.0f);
    const float p1 = w0;
    const float p2 = (q2 - c.g12 * p1) * c.ig22;
    const float p3 = (q3 - c.g1 * p1 - c.g2 * p2) * c.ig3;
    const float dl = w0 - wm1, dr = wp1 - w0;
    const float b1 = fminf(dl * dl, dr * dr);
    const float s2a = wm1 - 2.0f * w0 + wp1, s2b = wp1 - wm1;
    const float b2 = (13.0f / 12.0f) * s2a * s2a + 0.25f * s2b * s2b;
    const float o1 = 0.5f * (wp1 - wm1), o2 = 0.5f * (wp2 - wm2);
    // even part relative to w0 (beta ignores a constant added to the data)
    const float a1 = 0.5f * ((wp1 - w0) + (wm1 - w0)), a2 = 0.5f * ((wp2 - w0) + (wm2 - w0));
    const float c3 = (o2 - 2.0f * o1) * (1.0f / 6.0f);
    const float c1 = (34.0f * o1 - 5.0f * o2) * (1.0f / 24.0f);
    const float c4 = (a2 - 4.0f * a1) * (1.0f / 12.0f);
    const float c2 = (12.0f * a1 - a2) * 0.125f;
    const float b3 = c1 * (c1 + 0.5f * c3) + c2 * ((13.0f / 3.0f) * c2 + 4.2f * c4) + (3129.0f / 80.0f) * c3 * c3
                   + (87617.0f / 140.0f) * c4 * c4;
    const float t = 0.5f * (fabsf(b3 - b1) + fabsf(b3 - b2));
    const float tau = t * t;
    const float w1 = c.g1 * (1.0f + tau / (b1 + c.eps));
    const float w2 = c.g2 * (1.0f + tau / (b2 + c.eps));
    const float w3 = c.g3 * (1.0f + tau / (b3 + c.eps));
    return (w1 * p1 + w2 * p2 + w3 * p3) / (w1 + w2 + w3);
}

template <int DIM>
__device__ __forceinline__ void pair_flux_f(const float* S, int NB, int l, int r, float nx, float ny, float xt,
                                            const GasF& G, float* out) {
    const float rl = S[G_RHO * NB + l], rr = S[G_RHO * NB + r];
    const float Tl = S[G_T * NB + l], Tr = S[G_T * NB + r];
    const float rho_m = 0.5f * (rl + rr);
    const float T_m = 0.5f * (Tl + Tr);
    const float iT_m = 0.5f * (S[G_IT * NB + l] + S[G_IT * NB + r]);
    const float drho = (rl - rr) + (S[G_RHOL * NB + l] - S[G_RHOL * NB + r]);
    const float ilr = inv_log_mean_j(rl, rr, drho);
    const float ilT = inv_log_mean_j(Tl, Tr, (Tl - Tr) + (S[G_TL * NB + l] - S[G_TL * NB + r]));
    const float Pinv = S[G_IOM * NB + l] * S[G_IOM * NB + r];
    const float iTa = 1.0f / T_m;
    const float coef = G.Rb * Pinv - G.a * iTa;
    float D = G.R * ilr + coef - G.a * iTa;
    if (G.b > 0.0f) D += G.Rb * inv_log_mean_j(S[G_OM * NB + l], S[G_OM * NB + r], -G.b * drho);
    const float iD = 1.0f / D;
    const float g_m = 0.5f * (S[G_G * NB + l] + S[G_G * NB + r]);
    const float rT_m = 0.5f * (S[G_RT * NB + l] + S[G_RT * NB + r]);
    const float v2T_m = 0.5f * (S[G_V2T * NB + l] + S[G_V2T * NB + r]);
    const float vm1 = 0.5f * (S[G_V1 * NB + l] + S[G_V1 * NB + r]);
    const float vT1 = 0.5f * (S[G_VT1 * NB + l] + S[G_VT1 * NB + r]);
    const float rv1 = 0.5f * (S[G_RV1 * NB + l] + S[G_RV1 * NB + r]);
    const float U1 = (rho_m * coef + g_m) * iD;
    const float F11 = (rv1 * coef + g_m * vm1) * iD;
    const float P = rho_m * T_m * g_m;
    const float B0 = 0.5f * v2T_m - G.cv * T_m * ilT + 2.0f * G.a * rT_m;
    const float iiT = 1.0f / iT_m;
    if (DIM == 1) {
        const float Q1 = xt * U1 + nx * F11;
        const float sv = vT1 * vm1;
        out[0] = Q1;
        out[1] = vm1 * Q1 + nx * P;
        out[2] = (G.a * rT_m * (xt * rho_m + nx * rv1) + (sv - B0) * Q1 + P * nx * vT1) * iiT;
    } else {
        const float vm2 = 0.5f * (S[G_V2 * NB + l] + S[G_V2 * NB + r]);
        const float vT2 = 0.5f * (S[G_VT2 * NB + l] + S[G_VT2 * NB + r]);
        const float rv2 = 0.5f * (S[G_RV2 * NB + l] + S[G_RV2 * NB + r]);
        const float F21 = (rv2 * coef + g_m * vm2) * iD;
        const float Q1 = xt * U1 + nx * F11 + ny * F21;
        const float sv = vT1 * vm1 + vT2 * vm2;
        out[0] = Q1;
        out[1] = vm1 * Q1 + nx * P;
        out[2] = vm2 * Q1 + ny * P;
        out[3] = (G.a * rT_m * (xt * rho_m + nx * rv1 + ny * rv2) + (sv - B0) * Q1 + P * (nx * vT1 + ny * vT2)) * iiT;
    }
}

// Entropy-variable jump V_j - V_i written as the jump decomposition of Sec. 3.1
// (eq. jumpV) in general units, with every mean taken between nodes i and j:
//   [[V_1]] = [[rho]] (R/{rho}^ln + R b/{1-b rho}^ln + R b/Pi - 2a/{T})
//           + [[T]] (-c_v/{T}^ln + (2a {rho/T} + {|v|^2/T}/2)/{T}) - sum_m {v_m}[[v_m]]/{T}
//   [[V_{1+m}]] = ([[v_m]] - {v_m/T}[[T]])/{T},   [[V_E]] = [[T]]/(T_i T_j)
template <int DIM>
__device__ __forceinline__ void entropy_jump(const float* S, int NB, int i, int j, const GasF& G, float* dV) {
    const float ri = S[G_RHO * NB + i], rj = S[G_RHO * NB + j];
    const float Ti = S[G_T * NB + i], Tj = S[G_T * NB + j];
    // jumps from the double-float node values: exact hi difference plus lo difference
    const float dr = (rj - ri) + (S[G_RHOL * NB + j] - S[G_RHOL * NB + i]);
    const float dT = (Tj - Ti) + (S[G_TL * NB + j] - S[G_TL * NB + i]);
    const float iTa = 2.0f / (Ti + Tj);
    float crho = G.R * inv_log_mean_j(ri, rj, -dr) + G.Rb * S[G_IOM * NB + i] * S[G_IOM * NB + j] - 2.0f * G.a * iTa;
    if (G.b > 0.0f) crho += G.Rb * inv_log_mean_j(S[G_OM * NB + i], S[G_OM * NB + j], G.b * dr);
    const float rT = 0.5f * (S[G_RT * NB + i] + S[G_RT * NB + j]);
    const float v2T = 0.5f * (S[G_V2T * NB + i] + S[G_V2T * NB + j]);
    const float cT = -G.cv * inv_log_mean_j(Ti, Tj, -dT) + (2.0f * G.a * rT + 0.5f * v2T) * iTa;
    const float v1i = S[G_V1 * NB + i], v1j = S[G_V1 * NB + j];
    const float dv1 = (v1j - v1i) + (S[G_V1L * NB + j] - S[G_V1L * NB + i]);
    float kin = 0.5f * (v1i + v1j) * dv1;
    dV[1] = (dv1 - 0.5f * (S[G_VT1 * NB + i] + S[G_VT1 * NB + j]) * dT) * iTa;
    if (DIM == 2) {
        const float v2i = S[G_V2 * NB + i], v2j = S[G_V2 * NB + j];
        const float dv2 = (v2j - v2i) + (S[G_V2L * NB + j] - S[G_V2L * NB + i]);
        kin += 0.5f * (v2i + v2j) * dv2;
        dV[2] = (dv2 - 0.5f * (S[G_VT2 * NB + i] + S[G_VT2 * NB + j]) * dT) * iTa;
    }
    dV[0] = dr * crho + dT * cT - kin * iTa;
    dV[DIM + 1] = dT * S[G_IT * NB + i] * S[G_IT * NB + j];
}

// the face state of eq. HOstable's dissipation: log-mean density and pressure ratio, T, c, the rotation
// (cos, sin) of the face normal of length L, normal / tangential velocity, and the scalings of R^T T
struct FaceF {
    float rho, c, cs, sn, L, vn, vt, H, mid, sA, sE, sT, Lam, Hm, Hp;
};

template <int DIM>
__device__ __forceinline__ FaceF face_state_f(const float* S, int NB, int l, int step, float nx, float ny, float xtf,
                                              const GasF& G, DevStatus* st) {
    FaceF f;
    const int r = l + step;
    const float ilr = inv_log_mean_f(S[G_RHO * NB + l], S[G_RHO * NB + r]);
    const float rho = 1.0f / ilr;
    const float ilrp = inv_log_mean_f(S[G_RP * NB + l], S[G_RP * NB + r]);
    const float p = rho * ilrp;
    const float om = 1.0f - G.b * rho;
    const float T = (p + G.a * rho * rho) * om * ilr * G.iR;
    const float iom = 1.0f / om;
    const float c2 = (1.0f + G.delta) * G.R * T * iom * iom - 2.0f * G.a * rho;
    const float dcrit = G.R * T - 2.0f * G.a * rho * om * om;
    if (!(c2 > 0.0f) || !(dcrit > 0.0f) || !(om > 0.0f)) raise_error(st, ES_ERR_INADMISSIBLE, 0);
    const float c = sqrtf(c2);
    const float vm1 = 0.5f * (S[G_V1 * NB + l] + S[G_V1 * NB + r]);
    float cs = 1.0f, sn = 0.0f, L = 1.0f, vn = vm1, vt = 0.0f;
    if (DIM == 2) {
        const float vm2 = 0.5f * (S[G_V2 * NB + l] + S[G_V2 * NB + r]);
        L = sqrtf(nx * nx + ny * ny);
        const float iL = 1.0f / L;
        cs = nx * iL;
        sn = ny * iL;
        vn = cs * vm1 + sn * vm2;
        vt = -sn * vm1 + cs * vm2;
    } else {
        L = fabsf(nx);
        cs = nx > 0.0f ? 1.0f : -1.0f;
        vn = cs * vm1;
    }
    const float E = rho * (G.cv * T - G.a * rho) + 0.5f * rho * (vn * vn + vt * vt);
    const float H = (E + p) * ilr;
    f.rho = rho;
    f.c = c;
    f.cs = cs;
    f.sn = sn;
    f.L = L;
    f.vn = vn;
    f.vt = vt;
    f.H = H;
    f.mid = H - c2 * om * G.idelta;
    const float ic2 = 1.0f / c2;
    f.sA = sqrtf(0.5f * rho * T * ic2);
    f.sE = sqrtf(G.R * G.delta * rho * T * T * ic2 / dcrit);
    f.sT = sqrtf(rho * T);
    f.Lam = fabsf(xtf + L * vn) + L * c;
    f.Hm = H - vn * c;
    f.Hp = H + vn * c;
    return f;
}

template <int DIM>
__device__ __forceinline__ void face_dissipation_f(const float* S, int NB, int l, int step, float nx, float ny,
                                                   float xtf, const GasF& G, const WenoF& Wc, float* out,
                                                   DevStatus* st, const float* JB, int NJ, int jq) {
    const FaceF fs = face_state_f<DIM>(S, NB, l, step, nx, ny, xtf, G, st);
    const float c = fs.c, cs = fs.cs, sn = fs.sn, vn = fs.vn, vt = fs.vt, mid = fs.mid;
    const float sA = fs.sA, sE = fs.sE, sT = fs.sT, Lam = fs.Lam, Hm = fs.Hm, Hp = fs.Hp;

    // W_j - W_l = R^T T (V_j - V_l) at nodes l-2 .. l+3 (zero at l itself); V_j - V_l is the sum
    // of the neighbour jumps between them (JB[c][jq + q] = V_{q+1} - V_q along the line, the
    // face's left node at jq + 0)
    float W[6][DIM + 2];
    float aTV[DIM + 2];
    float cum[DIM + 2];
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) {
        W[2][m] = 0.0f;
        cum[m] = 0.0f;
    }
#pragma unroll
    for (int o = 3; o < 6; ++o)
#pragma unroll
        for (int m = 0; m < DIM + 2; ++m) {
            cum[m] += JB[m * NJ + jq + (o - 3)];
            W[o][m] = cum[m];
        }
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) cum[m] = 0.0f;
#pragma unroll
    for (int o = 1; o >= 0; --o)
#pragma unroll
        for (int m = 0; m < DIM + 2; ++m) {
            cum[m] -= JB[m * NJ + jq + (o - 2)];
            W[o][m] = cum[m];
        }
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        if (o == 2) continue;
        float dV[DIM + 2];
#pragma unroll
        for (int m = 0; m < DIM + 2; ++m) dV[m] = W[o][m];
        if (DIM == 1) {
            const float V0 = dV[0], V1 = cs * dV[1], V2 = dV[2];
            W[o][0] = sA * (V0 + (vn - c) * V1 + Hm * V2);
            W[o][1] = sE * (V0 + vn * V1 + mid * V2);
            W[o][2] = sA * (V0 + (vn + c) * V1 + Hp * V2);
            if (o == 3) {
                aTV[0] = fabsf(V0);
                aTV[1] = fabsf(V1);
                aTV[2] = fabsf(V2);
            }
        } else {
            const float V0 = dV[0];
            const float V1 = cs * dV[1] + sn * dV[2], V2 = -sn * dV[1] + cs * dV[2], V3 = dV[3];
            const float base = V0 + vt * V2;
            W[o][0] = sA * (base + (vn - c) * V1 + Hm * V3);
            W[o][1] = sE * (base + vn * V1 + mid * V3);
            W[o][2] = sT * (V2 + vt * V3);
            W[o][3] = sA * (base + (vn + c) * V1 + Hp * V3);
            if (o == 3) {
                aTV[0] = fabsf(V0);
                aTV[1] = fabsf(V1);
                aTV[2] = fabsf(V2);
                aTV[3] = fabsf(V3);
            }
        }
    }
    float scl[DIM + 2];
    if (DIM == 1) {
        scl[0] = sA * (aTV[0] + fabsf(vn - c) * aTV[1] + fabsf(Hm) * aTV[2]);
        scl[1] = sE * (aTV[0] + fabsf(vn) * aTV[1] + fabsf(mid) * aTV[2]);
        scl[2] = sA * (aTV[0] + fabsf(vn + c) * aTV[1] + fabsf(Hp) * aTV[2]);
    } else {
        const float avt = fabsf(vt);
        scl[0] = sA * (aTV[0] + fabsf(vn - c) * aTV[1] + avt * aTV[2] + fabsf(Hm) * aTV[3]);
        scl[1] = sE * (aTV[0] + fabsf(vn) * aTV[1] + avt * aTV[2] + fabsf(mid) * aTV[3]);
        scl[2] = sT * (aTV[2] + (avt + c) * aTV[3]);     // velocity round-off scales with |v_t| + c
        scl[3] = sA * (aTV[0] + fabsf(vn + c) * aTV[1] + avt * aTV[2] + fabsf(Hp) * aTV[3]);
    }
    float y[DIM + 2];
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) {
        const float wmin = mr_weno5_f(W[0][m], W[1][m], W[2][m], W[3][m], W[4][m], Wc);
        const float wplu = mr_weno5_f(W[5][m], W[4][m], W[3][m], W[2][m], W[1][m], Wc);
        const float jw = wplu - wmin;
        float j = W[3][m];
        if (fabsf(j) <= Wc.sign_tol * scl[m]) j = 0.0f;
        const bool keep = (jw > 0.0f && j > 0.0f) || (jw < 0.0f && j < 0.0f);
        y[m] = keep ? jw : 0.0f;
    }
    const float h = -0.5f * Lam;
    if (DIM == 1) {
        const float y0 = sA * y[0], y1 = sE * y[1], y2 = sA * y[2];
        out[0] = h * (y0 + y1 + y2);
        out[1] = h * cs * ((vn - c) * y0 + vn * y1 + (vn + c) * y2);
        out[2] = h * (Hm * y0 + mid * y1 + Hp * y2);
    } else {
        const float y0 = sA * y[0], y1 = sE * y[1], y2 = sT * y[2], y3 = sA * y[3];
        const float i0 = y0 + y1 + y3;
        const float i1 = (vn - c) * y0 + vn * y1 + (vn + c) * y3;
        const float i2 = vt * i0 + y2;
        const float i3 = Hm * y0 + mid * y1 + vt * y2 + Hp * y3;
        out[0] = h * i0;
        out[1] = h * (cs * i1 - sn * i2);
        out[2] = h * (sn * i1 + cs * i2);
        out[3] = h * i3;
    }
}

// face_dissipation_f in 2D shared by the two lanes (2 p, 2 p + 1) of a warp: both form the face state, lane
// half = 0 the characteristic components 0 and 1 (the acoustic wave u - c and the entropy wave), half = 1
// components 2 and 3 (the shear wave and u + c), each its own reconstructions and sign switch, and the two
// exchange their y values; every lane of the warp must call it (a lane without a face passes a valid one and
// drops the result).  The same arithmetic per component as face_dissipation_f; twice the lanes per face.
__device__ __forceinline__ void face_dissipation_split_f(const float* S, int NB, int l, int step, float nx, float ny,
                                                         float xtf, const GasF& G, const WenoF& Wc, float* out,
                                                         DevStatus* st, const float* JB, int NJ, int jq, int half) {
    const FaceF fs = face_state_f<2>(S, NB, l, step, nx, ny, xtf, G, st);
    const float c = fs.c, cs = fs.cs, sn = fs.sn, vn = fs.vn, vt = fs.vt, mid = fs.mid;
    const float sA = fs.sA, sE = fs.sE, sT = fs.sT, Lam = fs.Lam, Hm = fs.Hm, Hp = fs.Hp;
    const bool h0 = half == 0;
    // rows of R^T T for this lane's components: a = 0 or 2, b = 1 or 3; component 2 is sT (V2 + vt V3), the
    // others s (base + B V1 + D V3)
    const float s_a = h0 ? sA : sT, B_a = h0 ? vn - c : 0.0f, D_a = h0 ? Hm : vt;
    const float s_b = h0 ? sE : sA, B_b = h0 ? vn : vn + c, D_b = h0 ? mid : Hp;
    float Wa[6], Wb[6];
    float aTV[4];
    Wa[2] = 0.0f;
    Wb[2] = 0.0f;
    float cum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float Vn[6][4];
#pragma unroll
    for (int o = 3; o < 6; ++o)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            cum[m] += JB[m * NJ + jq + (o - 3)];
            Vn[o][m] = cum[m];
        }
#pragma unroll
    for (int m = 0; m < 4; ++m) cum[m] = 0.0f;
#pragma unroll
    for (int o = 1; o >= 0; --o)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            cum[m] -= JB[m * NJ + jq + (o - 2)];
            Vn[o][m] = cum[m];
        }
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        if (o == 2) continue;
        const float V0 = Vn[o][0];
        const float V1 = cs * Vn[o][1] + sn * Vn[o][2], V2 = -sn * Vn[o][1] + cs * Vn[o][2], V3 = Vn[o][3];
        const float base = V0 + vt * V2;
        Wa[o] = s_a * ((h0 ? base : V2) + B_a * V1 + D_a * V3);
        Wb[o] = s_b * (base + B_b * V1 + D_b * V3);
        if (o == 3) {
            aTV[0] = fabsf(V0);
            aTV[1] = fabsf(V1);
            aTV[2] = fabsf(V2);
            aTV[3] = fabsf(V3);
        }
    }
    const float avt = fabsf(vt);
    const float scl_a = h0 ? sA * (aTV[0] + fabsf(vn - c) * aTV[1] + avt * aTV[2] + fabsf(Hm) * aTV[3])
                           : sT * (aTV[2] + (avt + c) * aTV[3]);
    const float scl_b = s_b * (aTV[0] + fabsf(B_b) * aTV[1] + avt * aTV[2] + fabsf(D_b) * aTV[3]);
    float ya, yb;
    {
        const float wmin = mr_weno5_f(Wa[0], Wa[1], Wa[2], Wa[3], Wa[4], Wc);
        const float wplu = mr_weno5_f(Wa[5], Wa[4], Wa[3], Wa[2], Wa[1], Wc);
        const float jw = wplu - wmin;
        float j = Wa[3];
        if (fabsf(j) <= Wc.sign_tol * scl_a) j = 0.0f;
        const bool keep = (jw > 0.0f && j > 0.0f) || (jw < 0.0f && j < 0.0f);
        ya = keep ? jw : 0.0f;
    }
    {
        const float wmin = mr_weno5_f(Wb[0], Wb[1], Wb[2], Wb[3], Wb[4], Wc);
        const float wplu = mr_weno5_f(Wb[5], Wb[4], Wb[3], Wb[2], Wb[1], Wc);
        const float jw = wplu - wmin;
        float j = Wb[3];
        if (fabsf(j) <= Wc.sign_tol * scl_b) j = 0.0f;
        const bool keep = (jw > 0.0f && j > 0.0f) || (jw < 0.0f && j < 0.0f);
        yb = keep ? jw : 0.0f;
    }
    const float oa = __shfl_xor_sync(0xffffffffu, ya, 1);
    const float ob = __shfl_xor_sync(0xffffffffu, yb, 1);
    const float y[4] = {h0 ? ya : oa, h0 ? yb : ob, h0 ? oa : ya, h0 ? ob : yb};
    const float h = -0.5f * Lam;
    const float y0 = sA * y[0], y1 = sE * y[1], y2 = sT * y[2], y3 = sA * y[3];
    const float i0 = y0 + y1 + y3;
    const float i1 = (vn - c) * y0 + vn * y1 + (vn + c) * y3;
    const float i2 = vt * i0 + y2;
    const float i3 = Hm * y0 + mid * y1 + vt * y2 + Hp * y3;
    out[0] = h * i0;
    out[1] = h * (cs * i1 - sn * i2);
    out[2] = h * (sn * i1 + cs * i2);
    out[3] = h * i3;
}

template <int DIM>
__device__ __forceinline__ void load_node_f(float* S, int NB, int b, const StageParams& P, const GasF& G, int gi,
                                            int gj) {
    const int si = state_index(gi, P.n1, P.bc[0]);
    const int sj = DIM == 2 ? state_index(gj, P.n2, P.bc[1]) : 0;
    const int idx = sj * P.n1 + si;
    const size_t N = P.fcs;                                 // component stride
    const size_t LO = P.fps;                                // offset of the lo plane of JU
    // primitive state in double-float arithmetic
    const df iJ = df_recip({P.fJs[idx], P.fJs[P.fpsJ + idx]});
    const df rho = df_mul({P.fJUs[idx], P.fJUs[LO + idx]}, iJ);
    const df m1 = df_mul({P.fJUs[N + idx], P.fJUs[LO + N + idx]}, iJ);
    const df m2 = DIM == 2 ? df_mul({P.fJUs[2 * N + idx], P.fJUs[LO + 2 * N + idx]}, iJ) : df{0.0f, 0.0f};
    const df E = df_mul({P.fJUs[(DIM + 1) * N + idx], P.fJUs[LO + (DIM + 1) * N + idx]}, iJ);
    const df irho = df_recip(rho);
    const df v1 = df_mul(m1, irho);
    const df v2 = DIM == 2 ? df_mul(m2, irho) : df{0.0f, 0.0f};
    const df ke = df_mul_f(df_add(df_mul(v1, v1), df_mul(v2, v2)), 0.5f);
    // T = (E/rho - |v|^2/2 + a rho) / cv
    const df e = df_add(df_mul(E, irho), {-ke.hi, -ke.lo});
    const df Td = df_mul_f(df_add(e, df_mul_f(rho, G.a)), G.icv);
    const float r = rho.hi, T = Td.hi;
    const float om = 1.0f - G.b * r;
    const float iom = 1.0f / om;
    const float p = r * G.R * T * iom - G.a * r * r;
    const float iT = 1.0f / T;
    // what the node arithmetic needs; R T - 2 a rho (1 - b rho)^2 > 0 enters through the face states
    if (!(r > 0.0f) || !(om > 0.0f) || !(T > 0.0f) || !(p > 0.0f)) raise_error(P.status, ES_ERR_INADMISSIBLE, idx);
    S[G_RHO * NB + b] = r;
    S[G_RHOL * NB + b] = rho.lo;
    S[G_V1 * NB + b] = v1.hi;
    S[G_V1L * NB + b] = v1.lo;
    S[G_V2 * NB + b] = v2.hi;
    S[G_V2L * NB + b] = v2.lo;
    S[G_T * NB + b] = T;
    S[G_TL * NB + b] = Td.lo;
    S[G_IT * NB + b] = iT;
    S[G_OM * NB + b] = om;
    S[G_IOM * NB + b] = iom;
    S[G_G * NB + b] = G.R * iom - G.a * r * iT;
    S[G_RT * NB + b] = r * iT;
    S[G_VT1 * NB + b] = v1.hi * iT;
    S[G_VT2 * NB + b] = v2.hi * iT;
    S[G_V2T * NB + b] = 2.0f * ke.hi * iT;
    S[G_RV1 * NB + b] = m1.hi;
    S[G_RV2 * NB + b] = m2.hi;
    S[G_RP * NB + b] = r / p;
}

// FP32 displacement and mesh velocity at a possibly-ghost node: periodic wrap
// (the displacement is periodic), outflow odd reflection
template <int DIM>
__device__ __forceinline__ void stage_disp(const StageParams& P, int gi, int gj, float cdt, float* ds, float* xd) {
    const size_t N = P.fcs;
    if (gi >= 0 && gi < P.n1 && (DIM == 1 || (gj >= 0 && gj < P.n2))) {     // interior: plain loads
        const size_t id = size_t(DIM == 2 ? gj : 0) * P.n1 + gi;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const float xdk = P.fxdot ? P.fxdot[k * N + id] : 0.0f;
            ds[k] = P.fdisp[k * N + id] + cdt * xdk;
            xd[k] = xdk;
        }
        return;
    }
    const GhostTerms ti = ghost_terms(gi, P.n1, P.bc[0]);
    GhostTerms tj;
    if (DIM == 2) tj = ghost_terms(gj, P.n2, P.bc[1]);
    else { tj.idx[0] = 0; tj.w[0] = 1.0; tj.nterm = 1; tj.q = 0; }
    float acc[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int a = 0; a < ti.nterm; ++a)
        for (int c = 0; c < tj.nterm; ++c) {
            const float w = float(ti.w[a] * tj.w[c]);
            const size_t id = size_t(tj.idx[c]) * P.n1 + ti.idx[a];
            for (int k = 0; k < DIM; ++k) {
                const float xdk = P.fxdot ? P.fxdot[k * N + id] : 0.0f;
                acc[0][k] += w * (P.fdisp[k * N + id] + cdt * xdk);
                acc[1][k] += w * xdk;
            }
        }
    ds[0] = acc[0][0];
    xd[0] = acc[1][0];
    if (DIM == 2) {
        ds[1] = acc[0][1];
        xd[1] = acc[1][1];
    }
}


// One tile of the fused operator + RK stage (mixed form): the box of the tile at
// (i0, j0) is staged in shared memory S / PB / FB (TileF layout), then pair
// fluxes, face fluxes, divergence and the RK combination follow.  Called by the
// tiled kernel (one tile per CTA) and by the batched kernel (a loop over the
// chunks of one problem per CTA).
// SPLIT (2D): two lanes per face in the face phase (face_dissipation_split_f), for tiles with twice the threads
template <int DIM, int BX, int BY, int NT, bool SPLIT = false>
__device__ __forceinline__ void stage_tile_mixed(float* smemf, const StageParams& P, int i0, int j0, float dt,
                                                 const GasF& G, const WenoF& Wc) {
    static_assert(!SPLIT || DIM == 2, "the split face phase is written for 2D");
    using TL = TileF<DIM, BX, BY, NT>;
    constexpr int GX = TL::GX, NB = TL::NB, NC = TL::NC;
    float* S = smemf;
    float* PB = smemf + G_COUNT * NB;
    float* FB = PB + TL::PAIR_FLOATS;
    float* JB = FB + TL::NF * (NC + 1);
    const int tid = threadIdx.x;
    const float cdt = P.fcst * dt;
    const float idx1 = P.finv_dxi[0], idx2 = P.finv_dxi[1];
    float* XS = PB;
    float* XD = PB + 2 * NB;
    for (int b = tid; b < NB; b += NT) {
        const int ii = b % GX, jj = b / GX;
        const int gi = i0 - 3 + ii, gj = j0 - 3 + jj;
        float ds[2], xd[2];
        stage_disp<DIM>(P, gi, DIM == 2 ? gj : 0, cdt, ds, xd);
        XS[b] = ds[0];
        XD[b] = xd[0];
        if (DIM == 2) {
            XS[NB + b] = ds[1];
            XD[NB + b] = xd[1];
        }
        const bool in_x = ii >= 3 && ii < 3 + BX;
        const bool in_y = DIM == 1 || (jj >= 3 && jj < 3 + BY);
        if (in_x || in_y) load_node_f<DIM>(S, NB, b, P, G, gi, gj);
    }
    __syncthreads();
    for (int b = tid; b < NB; b += NT) {
        const int ii = b % GX, jj = b / GX;
        if (DIM == 1) {
            S[G_N1X * NB + b] = 1.0f;
            S[G_N1Y * NB + b] = 0.0f;
            S[G_XT1 * NB + b] = -XD[b];
        } else {
            if (jj >= 3 && jj < 3 + BY) {        // J dxi_1/dx = (1 + d2[d_y]/dxi_2, -d2[d_x]/dxi_2)
                float dy = 0.0f, dx = 0.0f;
#pragma unroll
                for (int m = 1; m <= 3; ++m) {
                    const float h = 0.5f * float(ec_alpha(m));
                    dx += h * (XS[b + m * GX] - XS[b - m * GX]);
                    dy += h * (XS[NB + b + m * GX] - XS[NB + b - m * GX]);
                }
                const float nx = 1.0f + dy * idx2, ny = -dx * idx2;
                S[G_N1X * NB + b] = nx;
                S[G_N1Y * NB + b] = ny;
                S[G_XT1 * NB + b] = -(XD[b] * nx + XD[NB + b] * ny);
            }
            if (ii >= 3 && ii < 3 + BX) {        // J dxi_2/dx = (-d1[d_y]/dxi_1, 1 + d1[d_x]/dxi_1)
                float dy = 0.0f, dx = 0.0f;
#pragma unroll
                for (int m = 1; m <= 3; ++m) {
                    const float h = 0.5f * float(ec_alpha(m));
                    dx += h * (XS[b + m] - XS[b - m]);
                    dy += h * (XS[NB + b + m] - XS[NB + b - m]);
                }
                const float nx = -dy * idx1, ny = 1.0f + dx * idx1;
                S[G_N2X * NB + b] = nx;
                S[G_N2Y * NB + b] = ny;
                S[G_XT2 * NB + b] = -(XD[b] * nx + XD[NB + b] * ny);
            }
        }
    }
    __syncthreads();

    float acc[NC + 1];
#pragma unroll
    for (int c = 0; c <= NC; ++c) acc[c] = 0.0f;
    const int tx = tid % BX, ty = tid / BX;

    // one copy of the direction pipeline for both directions (unrolled, the kernel's code was twice the size
    // and its warps stalled on instruction fetch); the line lengths and strides are then run-time values
#pragma unroll 1
    for (int k = 0; k < DIM; ++k) {
        const int nlines = k == 0 ? (DIM == 2 ? BY : 1) : BX;
        const int LB = k == 0 ? BX : BY;
        const int per_line = 3 * LB + 6;
        const int step = k == 0 ? 1 : GX;
        const int fN = k == 0 ? G_N1X : G_N2X;
        const int fNy = k == 0 ? G_N1Y : G_N2Y;
        const int fXT = k == 0 ? G_XT1 : G_XT2;
        for (int t = tid; t < nlines * per_line; t += NT) {
            const int line = t / per_line, kk = t % per_line;
            int m, q;
            if (kk < LB + 1) { m = 1; q = 2 + kk; }
            else if (kk < 2 * LB + 3) { m = 2; q = 1 + (kk - LB - 1); }
            else { m = 3; q = kk - 2 * LB - 3; }
            const int base = k == 0 ? (DIM == 2 ? (3 + line) * GX : 0) : 3 + line;
            const int l = base + q * step, r = l + m * step;
            const float nx = 0.5f * (S[fN * NB + l] + S[fN * NB + r]);
            const float ny = 0.5f * (S[fNy * NB + l] + S[fNy * NB + r]);
            const float xt = 0.5f * (S[fXT * NB + l] + S[fXT * NB + r]);
            float f[NC];
            pair_flux_f<DIM>(S, NB, l, r, nx, ny, xt, G, f);
#pragma unroll
            for (int c = 0; c < NC; ++c) PB[c * TL::NP + t] = f[c];
        }
        if (P.diss) {
            // neighbour jumps V_{q+1} - V_q, q = 0 .. LB+4 along each line (eq. jumpV)
            for (int t = tid; t < nlines * (LB + 5); t += NT) {
                const int line = t / (LB + 5), q = t % (LB + 5);
                const int base = k == 0 ? (DIM == 2 ? (3 + line) * GX : 0) : 3 + line;
                const int l = base + q * step;
                float dV[NC];
                entropy_jump<DIM>(S, NB, l, l + step, G, dV);
#pragma unroll
                for (int c = 0; c < NC; ++c) JB[c * TL::NJ + t] = dV[c];
            }
        }
        __syncthreads();
        const int nfaces = nlines * (LB + 1);
        const int lane = tid & 31;
        // SPLIT: lanes (2 p, 2 p + 1) share face p; the trip count is uniform per warp (the halves exchange
        // values), and a lane past the last face works on the last face and stores nothing
        for (int ub = SPLIT ? tid - lane : tid; ub < (SPLIT ? 2 * nfaces : nfaces); ub += NT) {
            const int u = SPLIT ? ub + lane : ub;
            const bool active = !SPLIT || u < 2 * nfaces;
            const int t = SPLIT ? (active ? (u >> 1) : nfaces - 1) : u;
            const int half = SPLIT ? (u & 1) : 0;
            const int line = t / (LB + 1), f = t % (LB + 1);
            const int q = 2 + f;
            const int pbase = line * per_line;
            float F[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) F[c] = 0.0f;
            float FJ = 0.0f;
            const int base = k == 0 ? (DIM == 2 ? (3 + line) * GX : 0) : 3 + line;
#pragma unroll
            for (int m = 1; m <= 3; ++m) {
                const int off = m == 1 ? 0 : (m == 2 ? LB + 1 : 2 * LB + 3);
                const float al = float(ec_alpha(m));
                for (int s = 0; s < m; ++s) {
                    const int qq = q - s;
                    const int pi = pbase + off + (qq - (3 - m));
#pragma unroll
                    for (int c = 0; c < NC; ++c) F[c] += al * PB[c * TL::NP + pi];
                    FJ += al * 0.5f * (S[fXT * NB + base + qq * step] + S[fXT * NB + base + (qq + m) * step]);
                }
            }
            if (P.diss) {
                const int l = base + q * step;
                const float nx = 0.5f * (S[fN * NB + l] + S[fN * NB + l + step]);
                const float ny = 0.5f * (S[fNy * NB + l] + S[fNy * NB + l + step]);
                const float xtf = 0.5f * (S[fXT * NB + l] + S[fXT * NB + l + step]);
                float d[NC];
                if constexpr (SPLIT)
                    face_dissipation_split_f(S, NB, l, step, nx, ny, xtf, G, Wc, d, P.status, JB, TL::NJ,
                                             line * (LB + 5) + q, half);
                else
                    face_dissipation_f<DIM>(S, NB, l, step, nx, ny, xtf, G, Wc, d, P.status, JB, TL::NJ,
                                            line * (LB + 5) + q);
#pragma unroll
                for (int c = 0; c < NC; ++c) F[c] += d[c];
            }
            if (active && half == 0) {
#pragma unroll
                for (int c = 0; c < NC; ++c) FB[c * TL::NF + t] = F[c];
                FB[NC * TL::NF + t] = FJ;
            }
        }
        __syncthreads();
        if (tid < BX * (DIM == 2 ? BY : 1)) {
            const int line = k == 0 ? ty : tx;
            const int pos = k == 0 ? tx : ty;
            const int fm = line * (LB + 1) + pos;
            const float inv = k == 0 ? idx1 : idx2;
#pragma unroll
            for (int c = 0; c <= NC; ++c) acc[c] -= (FB[c * TL::NF + fm + 1] - FB[c * TL::NF + fm]) * inv;
        }
        __syncthreads();
    }

    const int gi = i0 + tx, gj = j0 + ty;
    if (tid < BX * (DIM == 2 ? BY : 1) && gi < P.n1 && (DIM == 1 || gj < P.n2)) {
        const size_t N = P.fcs;
        const size_t idx = size_t(DIM == 2 ? gj : 0) * P.n1 + gi;
        const size_t LO = P.fps;
        if (P.mode == 1) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                P.fJUo[c * N + idx] = acc[c];
                P.fJUo[LO + c * N + idx] = 0.0f;
            }
            P.fJo[idx] = acc[NC];
            P.fJo[P.fpsJ + idx] = 0.0f;
        } else {
            // a_s U^n + b_s (U^s + dt L) in double-float (a_s, b_s are 0, 1, 3/4, 1/4, 1/3, 2/3)
            const float ca = P.fca, cb = P.fcb;
            const float ca_lo = P.fca_lo, cb_lo = P.fcb_lo;
            // all operands loaded before the first store: as far as the compiler knows a store may alias a
            // later load, which would serialise one round trip per component
            df Un[NC + 1], Us[NC + 1];
#pragma unroll
            for (int c = 0; c <= NC; ++c) {
                const float* un = c < NC ? P.fJUn + c * N : P.fJn;
                const float* us = c < NC ? P.fJUs + c * N : P.fJs;
                const size_t lo = c < NC ? LO : P.fpsJ;
                Us[c] = {us[idx], us[lo + idx]};
                Un[c] = ca != 0.0f ? df{un[idx], un[lo + idx]} : df{0.0f, 0.0f};
            }
#pragma unroll
            for (int c = 0; c <= NC; ++c) {
                float* uo = c < NC ? P.fJUo + c * N : P.fJo;
                const size_t lo = c < NC ? LO : P.fpsJ;
                const df inc = df_add_f(Us[c], dt * acc[c]);
                df outv = df_mul(inc, {cb, cb_lo});
                if (ca != 0.0f) outv = df_add(outv, df_mul(Un[c], {ca, ca_lo}));
                uo[idx] = outv.hi;
                uo[lo + idx] = outv.lo;
                if (c == NC && !(outv.hi > 0.0f)) raise_error(P.status, ES_ERR_MESH, int(idx));
            }
        }
    }
}

// float copies of the gas and WENO constants of a launch
__device__ __forceinline__ GasF gas_f(const StageParams& P) {
    GasF G;
    G.a = P.fgas[0];
    G.b = P.fgas[1];
    G.R = P.fgas[2];
    G.cv = P.fgas[3];
    G.delta = P.fgas[4];
    G.Rb = P.fgas[5];
    G.icv = P.fgas[6];
    G.iR = P.fgas[7];
    G.idelta = P.fgas[8];
    return G;
}

__device__ __forceinline__ WenoF weno_f(const StageParams& P) {
    WenoF W;
    W.g1 = P.fweno[0];
    W.g2 = P.fweno[1];
    W.g3 = P.fweno[2];
    W.g12 = P.fweno[3];
    W.ig22 = P.fweno[4];
    W.ig3 = P.fweno[5];
    W.eps = P.fweno[6];
    W.sign_tol = P.fweno[7];
    return W;
}

}  // namespace mixed
}  // namespace es
