// es_stage.cu -- fused semi-discrete ES operator + SSP-RK3 stage, FP64 form.
//
// One CTA owns a BX x BY tile of nodes (BY = 1 in 1D).  It stages a box with
// a 3-node halo in shared memory (the reach of the 6-point pair stencil and of
// WENO5), computes per node the primitive state, logarithms and entropy
// variables once, the metrics of the stage mesh (Sec. 3.2, eq. SCLCoeff and
// VCLCoeff), then per direction:
//   pair fluxes F(U_q, U_{q+m}), m = 1..3 (Sec. 3.1, eq. ECfluxMM), shared
//   by the faces that use them,
//   face fluxes = the 6th-order combination (eq. ECFlux_curv_2p, GCL_flux)
//   plus the ES dissipation (eq. HOstable) with MR-WENO5 on the scaled
//   entropy variables,
//   the divergence (eq. semi_U, semi_J),
// and finally the Shu-Osher SSP-RK3 combination.  Nothing but the inputs and
// the outputs touches global memory.
#include <cuda_runtime.h>

#include "es_device.cuh"
#include "es_internal.h"

namespace es {

// shared-memory field slots (each NB doubles)
enum Field {
    F_RHO, F_V1, F_V2, F_T, F_IT, F_OM, F_IOM, F_G, F_RT, F_VT1, F_VT2, F_V2T, F_RV1, F_RV2,
    F_LNR, F_LNOM, F_LNT, F_RP, F_LNRP, F_W0, F_W1, F_W2, F_W3,
    F_N1X, F_N1Y, F_XT1, F_N2X, F_N2Y, F_XT2,
    F_COUNT
};

template <int DIM, int BX, int BY, int NT>
struct Tile {
    static constexpr int GX = BX + 6;
    static constexpr int GY = DIM == 2 ? BY + 6 : 1;
    static constexpr int NB = GX * GY;
    static constexpr int NC = DIM + 2;
    static constexpr int ROWP = 3 * BX + 6;                 // pairs per xi_1 line
    static constexpr int COLP = 3 * BY + 6;                 // pairs per xi_2 line
    static constexpr int NP1 = (DIM == 2 ? BY : 1) * ROWP;
    static constexpr int NP2 = DIM == 2 ? BX * COLP : 0;
    static constexpr int NP = NP1 > NP2 ? NP1 : NP2;
    static constexpr int NF1 = (DIM == 2 ? BY : 1) * (BX + 1);
    static constexpr int NF2 = DIM == 2 ? BX * (BY + 1) : 0;
    static constexpr int NF = NF1 > NF2 ? NF1 : NF2;
    // Joint schedule (2D, when shared memory allows): the pairs of both directions in one phase
    // and their faces in the next (two block barriers per stage instead of six, and the faces
    // dealt to the warps as one pool of NF1 + NF2).  Otherwise pairs and faces go direction by
    // direction.
    static constexpr size_t FIELDS = sizeof(double) * size_t(F_COUNT) * NB;
    static constexpr int PAIRJ = ((NP1 + NP2) * NC > 4 * NB) ? (NP1 + NP2) * NC : 4 * NB;
    static constexpr size_t SMEM_JOINT = FIELDS + sizeof(double) * (size_t(PAIRJ) + size_t(NF1 + NF2) * (NC + 1));
    static constexpr bool JOINT = DIM == 2 && SMEM_JOINT <= 227 * 1024;
    // pair and face buffers: per-component strides and the offset of direction 2's entries
    static constexpr int PS = JOINT ? NP1 + NP2 : NP;
    static constexpr int FS = JOINT ? NF1 + NF2 : NF;
    static constexpr int POFF2 = JOINT ? NP1 : 0;
    static constexpr int FOFF2 = JOINT ? NF1 : 0;
    static constexpr int PAIR_DOUBLES = JOINT ? PAIRJ : ((NP * NC > 4 * NB) ? NP * NC : 4 * NB);   // also holds coords
    static constexpr size_t SMEM = FIELDS + sizeof(double) * (size_t(PAIR_DOUBLES) + size_t(FS) * (NC + 1));
    static constexpr int THREADS = NT;
    static_assert(NT >= BX * (DIM == 2 ? BY : 1) && NT % 32 == 0, "threads cover the tile");
};

// --------------------------------------------------------------- pair flux
// Two-point EC flux of Sec. 3.1 contracted with the face-averaged metrics:
//   F = {J xi_t} U~ + sum_j {J xi_k/x_j} F~_j,
// U~, F~_j from the explicit solution of eq. linear_U / linear_F in general
// units (D U~_1 = {rho}(Rb/Pi - a/{T}) + {g}, U~_{1+m} = {v_m} U~_1, ...).
template <int DIM>
__device__ __forceinline__ void pair_flux(const double* S, int NB, int l, int r, double nx, double ny,
                                          double xt, const Gas& G, double* out) {
    const double* rho = S + F_RHO * NB;
    const double rl = rho[l], rr = rho[r];
    const double Tl = S[F_T * NB + l], Tr = S[F_T * NB + r];
    const double rho_m = 0.5 * (rl + rr);
    const double T_m = 0.5 * (Tl + Tr);
    const double iT_m = 0.5 * (S[F_IT * NB + l] + S[F_IT * NB + r]);
    const double ilr = inv_log_mean(rl, rr, S[F_LNR * NB + l], S[F_LNR * NB + r]);
    const double ilT = inv_log_mean(Tl, Tr, S[F_LNT * NB + l], S[F_LNT * NB + r]);
    const double Pinv = S[F_IOM * NB + l] * S[F_IOM * NB + r];
    const double iTa = rcp_nr(T_m);
    const double coef = G.R * G.b * Pinv - G.a * iTa;
    double D = G.R * ilr + coef - G.a * iTa;
    if (G.b > 0.0)
        D += G.R * G.b * inv_log_mean(S[F_OM * NB + l], S[F_OM * NB + r], S[F_LNOM * NB + l], S[F_LNOM * NB + r]);
    const double iD = rcp_nr(D);
    const double g_m = 0.5 * (S[F_G * NB + l] + S[F_G * NB + r]);
    const double rT_m = 0.5 * (S[F_RT * NB + l] + S[F_RT * NB + r]);
    const double v2T_m = 0.5 * (S[F_V2T * NB + l] + S[F_V2T * NB + r]);
    const double vm1 = 0.5 * (S[F_V1 * NB + l] + S[F_V1 * NB + r]);
    const double vT1 = 0.5 * (S[F_VT1 * NB + l] + S[F_VT1 * NB + r]);
    const double rv1 = 0.5 * (S[F_RV1 * NB + l] + S[F_RV1 * NB + r]);
    const double U1 = (rho_m * coef + g_m) * iD;
    const double F11 = (rv1 * coef + g_m * vm1) * iD;
    const double P = rho_m * T_m * g_m;
    const double B0 = 0.5 * v2T_m - G.cv * T_m * ilT + 2.0 * G.a * rT_m;
    if (DIM == 1) {
        const double Q1 = xt * U1 + nx * F11;
        const double sv = vT1 * vm1;
        out[0] = Q1;
        out[1] = vm1 * Q1 + nx * P;
        out[2] = div_nr(G.a * rT_m * (xt * rho_m + nx * rv1) + (sv - B0) * Q1 + P * nx * vT1, iT_m);
    } else {
        const double vm2 = 0.5 * (S[F_V2 * NB + l] + S[F_V2 * NB + r]);
        const double vT2 = 0.5 * (S[F_VT2 * NB + l] + S[F_VT2 * NB + r]);
        const double rv2 = 0.5 * (S[F_RV2 * NB + l] + S[F_RV2 * NB + r]);
        const double F21 = (rv2 * coef + g_m * vm2) * iD;
        const double Q1 = xt * U1 + nx * F11 + ny * F21;
        const double sv = vT1 * vm1 + vT2 * vm2;
        out[0] = Q1;
        out[1] = vm1 * Q1 + nx * P;
        out[2] = vm2 * Q1 + ny * P;
        out[3] = div_nr(G.a * rT_m * (xt * rho_m + nx * rv1 + ny * rv2) + (sv - B0) * Q1 + P * (nx * vT1 + ny * vT2),
                        iT_m);
    }
}

// -------------------------------------------------------- ES dissipation
// -1/2 Lambda T^{-1} R Y [[W]]^WENO at the face between box nodes l and l+step
// (Sec. 3.3, eq. HOstable).  Face state rho = {rho}^ln, v = {v}, p = {rho}^ln/{rho/p}^ln;
// face metrics and J xi_t are means of the two node values; R = R~ S in the frame
// rotated to the face normal; W = R^T T V at the six stencil nodes.
template <int DIM>
__device__ __forceinline__ void face_dissipation(const double* S, int NB, int l, int step, double nx, double ny,
                                                 double xtf, const Gas& G, const Weno& Wc, double* out,
                                                 DevStatus* st, int gidx) {
    const int r = l + step;
    const double ilr = inv_log_mean(S[F_RHO * NB + l], S[F_RHO * NB + r], S[F_LNR * NB + l], S[F_LNR * NB + r]);
    const double rho = rcp_nr(ilr);
    const double ilrp = inv_log_mean(S[F_RP * NB + l], S[F_RP * NB + r], S[F_LNRP * NB + l], S[F_LNRP * NB + r]);
    const double p = rho * ilrp;
    const double om = 1.0 - G.b * rho;
    const double T = (p + G.a * rho * rho) * om * ilr * G.iR;
    const double iom = rcp_nr(om);
    const double c2 = (1.0 + G.delta) * G.R * T * iom * iom - 2.0 * G.a * rho;
    const double dcrit = G.R * T - 2.0 * G.a * rho * om * om;
    if (!(c2 > 0.0) || !(dcrit > 0.0) || !(om > 0.0)) raise_error(st, ES_ERR_INADMISSIBLE, gidx);
    const double c = sqrt(c2);
    const double vm1 = 0.5 * (S[F_V1 * NB + l] + S[F_V1 * NB + r]);
    double cs = 1.0, sn = 0.0, L = 1.0, vn = vm1, vt = 0.0;
    if (DIM == 2) {
        const double vm2 = 0.5 * (S[F_V2 * NB + l] + S[F_V2 * NB + r]);
        L = sqrt(nx * nx + ny * ny);
        const double iL = rcp_nr(L);
        cs = nx * iL;
        sn = ny * iL;
        vn = cs * vm1 + sn * vm2;
        vt = -sn * vm1 + cs * vm2;
    } else {
        L = fabs(nx);
        cs = nx > 0.0 ? 1.0 : -1.0;
        vn = cs * vm1;
    }
    const double E = rho * (G.cv * T - G.a * rho) + 0.5 * rho * (vn * vn + vt * vt);
    const double H = (E + p) * ilr;
    const double mid = H - c2 * om * G.idelta;
    const double ic2 = rcp_nr(c2);
    const double sA = sqrt(0.5 * rho * T * ic2);
    const double sE = sqrt(div_nr(G.R * G.delta * rho * T * T * ic2, dcrit));
    const double sT = sqrt(rho * T);
    const double Lam = fabs(xtf + L * vn) + L * c;
    const double Hm = H - vn * c, Hp = H + vn * c;

    // scaled entropy variables W = R^T (T V) at nodes l-2 .. l+3; aTV = |T V_i| + |T V_{i+1}|
    double W[6][DIM + 2];
    double aTV[DIM + 2];
#pragma unroll
    for (int a = 0; a < DIM + 2; ++a) aTV[a] = 0.0;
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        const int q = l + (o - 2) * step;
        const double V0 = S[F_W0 * NB + q];
        if (DIM == 1) {
            const double V1 = cs * S[F_W1 * NB + q], V2 = S[F_W2 * NB + q];
            W[o][0] = sA * (V0 + (vn - c) * V1 + Hm * V2);
            W[o][1] = sE * (V0 + vn * V1 + mid * V2);
            W[o][2] = sA * (V0 + (vn + c) * V1 + Hp * V2);
            if (o == 2 || o == 3) {
                aTV[0] += fabs(V0);
                aTV[1] += fabs(V1);
                aTV[2] += fabs(V2);
            }
        } else {
            const double a1 = S[F_W1 * NB + q], a2 = S[F_W2 * NB + q];
            const double V1 = cs * a1 + sn * a2, V2 = -sn * a1 + cs * a2, V3 = S[F_W3 * NB + q];
            const double base = V0 + vt * V2;
            W[o][0] = sA * (base + (vn - c) * V1 + Hm * V3);
            W[o][1] = sE * (base + vn * V1 + mid * V3);
            W[o][2] = sT * (V2 + vt * V3);
            W[o][3] = sA * (base + (vn + c) * V1 + Hp * V3);
            if (o == 2 || o == 3) {
                aTV[0] += fabs(V0);
                aTV[1] += fabs(V1);
                aTV[2] += fabs(V2);
                aTV[3] += fabs(V3);
            }
        }
    }
    // round-off size of each W_m: sum_a |R_am| aTV_a
    double scl[DIM + 2];
    if (DIM == 1) {
        scl[0] = sA * (aTV[0] + fabs(vn - c) * aTV[1] + fabs(Hm) * aTV[2]);
        scl[1] = sE * (aTV[0] + fabs(vn) * aTV[1] + fabs(mid) * aTV[2]);
        scl[2] = sA * (aTV[0] + fabs(vn + c) * aTV[1] + fabs(Hp) * aTV[2]);
    } else {
        const double avt = fabs(vt);
        scl[0] = sA * (aTV[0] + fabs(vn - c) * aTV[1] + avt * aTV[2] + fabs(Hm) * aTV[3]);
        scl[1] = sE * (aTV[0] + fabs(vn) * aTV[1] + avt * aTV[2] + fabs(mid) * aTV[3]);
        scl[2] = sT * (aTV[2] + (avt + c) * aTV[3]);     // velocity round-off scales with |v_t| + c
        scl[3] = sA * (aTV[0] + fabs(vn + c) * aTV[1] + avt * aTV[2] + fabs(Hp) * aTV[3]);
    }
    double y[DIM + 2];
#pragma unroll
    for (int m = 0; m < DIM + 2; ++m) {
        const double wmin = mr_weno5(W[0][m], W[1][m], W[2][m], W[3][m], W[4][m], Wc);
        const double wplu = mr_weno5(W[5][m], W[4][m], W[3][m], W[2][m], W[1][m], Wc);
        const double jw = wplu - wmin;
        double j = W[3][m] - W[2][m];
        if (fabs(j) <= Wc.sign_tol * scl[m]) j = 0.0;     // round-off of a zero jump: sign 0
        const bool keep = (jw > 0.0 && j > 0.0) || (jw < 0.0 && j < 0.0);
        y[m] = keep ? jw : 0.0;
    }
    const double h = -0.5 * Lam;
    if (DIM == 1) {
        const double y0 = sA * y[0], y1 = sE * y[1], y2 = sA * y[2];
        out[0] = h * (y0 + y1 + y2);
        out[1] = h * cs * ((vn - c) * y0 + vn * y1 + (vn + c) * y2);
        out[2] = h * (Hm * y0 + mid * y1 + Hp * y2);
    } else {
        const double y0 = sA * y[0], y1 = sE * y[1], y2 = sT * y[2], y3 = sA * y[3];
        const double i0 = y0 + y1 + y3;
        const double i1 = (vn - c) * y0 + vn * y1 + (vn + c) * y3;
        const double i2 = vt * i0 + y2;
        const double i3 = Hm * y0 + mid * y1 + vt * y2 + Hp * y3;
        out[0] = h * i0;
        out[1] = h * (cs * i1 - sn * i2);
        out[2] = h * (sn * i1 + cs * i2);
        out[3] = h * i3;
    }
}

// ----------------------------------------------------------- node loader
template <int DIM>
__device__ __forceinline__ void load_node(double* S, int NB, int b, const StageParams& P, int gi, int gj) {
    const Gas& G = P.gas;
    const int si = state_index(gi, P.n1, P.bc[0]);
    const int sj = DIM == 2 ? state_index(gj, P.n2, P.bc[1]) : 0;
    const int idx = sj * P.n1 + si;
    const size_t N = size_t(P.n1) * P.n2;
    const double iJ = rcp_nr(P.Js[idx]);
    const double rho = P.JUs[idx] * iJ;
    // at a wall or symmetry end the ghost is the mirror node with the normal momentum negated
    const double f1 = (gi < 0 || gi >= P.n1) && end_mirrored(P.bc[0], gi < 0) ? -1.0 : 1.0;
    const double f2 = DIM == 2 && (gj < 0 || gj >= P.n2) && end_mirrored(P.bc[1], gj < 0) ? -1.0 : 1.0;
    const double m1 = f1 * (P.JUs[N + idx] * iJ);
    const double m2 = DIM == 2 ? f2 * (P.JUs[2 * N + idx] * iJ) : 0.0;
    const double E = P.JUs[(DIM + 1) * N + idx] * iJ;
    const double irho = rcp_nr(rho);
    const double v1 = m1 * irho, v2 = m2 * irho;
    const double ke = 0.5 * (v1 * v1 + v2 * v2);
    const double T = (E * irho - ke + G.a * rho) * G.icv;
    const double om = 1.0 - G.b * rho;
    const double iom = rcp_nr(om);
    const double p = rho * G.R * T * iom - G.a * rho * rho;
    const double iT = rcp_nr(T);
    // what the node arithmetic needs (logarithms of rho, 1 - b rho, T, p); the
    // condition R T - 2 a rho (1 - b rho)^2 > 0 enters through the face states
    if (!(rho > 0.0) || !(om > 0.0) || !(T > 0.0) || !(p > 0.0)) raise_error(P.status, ES_ERR_INADMISSIBLE, idx);
    const double lnr = log(rho);
    const double lnom = G.b > 0.0 ? log(om) : 0.0;
    const double lnT = log(T);
    const double lnp = log(p);
    S[F_RHO * NB + b] = rho;
    S[F_V1 * NB + b] = v1;
    S[F_V2 * NB + b] = v2;
    S[F_T * NB + b] = T;
    S[F_IT * NB + b] = iT;
    S[F_OM * NB + b] = om;
    S[F_IOM * NB + b] = iom;
    S[F_G * NB + b] = G.R * iom - G.a * rho * iT;
    S[F_RT * NB + b] = rho * iT;
    S[F_VT1 * NB + b] = v1 * iT;
    S[F_VT2 * NB + b] = v2 * iT;
    S[F_V2T * NB + b] = 2.0 * ke * iT;
    S[F_RV1 * NB + b] = m1;
    S[F_RV2 * NB + b] = m2;
    S[F_LNR * NB + b] = lnr;
    S[F_LNOM * NB + b] = lnom;
    S[F_LNT * NB + b] = lnT;
    S[F_RP * NB + b] = div_nr(rho, p);
    S[F_LNRP * NB + b] = lnr - lnp;
    // entropy variables V = ((e + p/rho)/T - s - |v|^2/(2T), v/T, -1/T), s = cv ln T + R ln((1 - b rho)/rho)
    const double s = G.cv * lnT + G.R * (lnom - lnr);
    S[F_W0 * NB + b] = G.cv - s - 2.0 * G.a * rho * iT + G.R * iom - ke * iT;
    S[F_W1 * NB + b] = v1 * iT;
    if (DIM == 2) {
        S[F_W2 * NB + b] = v2 * iT;
        S[F_W3 * NB + b] = -iT;
    } else {
        S[F_W2 * NB + b] = -iT;
    }
}

// stage coordinates x^n + c dt xdot and mesh velocity at a possibly-ghost node
template <int DIM>
__device__ __forceinline__ void stage_coords(const StageParams& P, int gi, int gj, double cdt, double* xs,
                                             double* xd) {
    const size_t N = size_t(P.n1) * P.n2;
    // per component k: a wall or symmetry end mirrors the components along it (tangential) and
    // reflects the normal one; the other ends treat every component alike
    for (int k = 0; k < DIM; ++k) {
        const GhostTerms ti = ghost_terms(gi, P.n1, P.bc[0], k != 0);
        GhostTerms tj;
        if (DIM == 2) tj = ghost_terms(gj, P.n2, P.bc[1], k != 1);
        else { tj.idx[0] = 0; tj.w[0] = 1.0; tj.nterm = 1; tj.q = 0; }
        double as = 0.0, ad = 0.0;
        for (int a = 0; a < ti.nterm; ++a)
            for (int c = 0; c < tj.nterm; ++c) {
                const double w = ti.w[a] * tj.w[c];
                const size_t id = size_t(tj.idx[c]) * P.n1 + ti.idx[a];
                const double xdk = P.xdot ? P.xdot[k * N + id] : 0.0;
                as += w * (P.xn[k * N + id] + cdt * xdk);
                ad += w * xdk;
            }
        xs[k] = as + (k == 0 ? ti.q * P.period[0] : tj.q * P.period[1]);
        xd[k] = ad;
    }
}

// geometry of direction k in the box: lines, interior nodes per line, pairs per line, node step
// and the metric slots
template <int DIM, int BX, int BY>
struct DirGeo {
    int k, nlines, LB, per_line, step, fN, fNy, fXT;
    __device__ __forceinline__ explicit DirGeo(int kk) : k(kk) {
        nlines = k == 0 ? (DIM == 2 ? BY : 1) : BX;
        LB = k == 0 ? BX : BY;
        per_line = 3 * LB + 6;
        step = k == 0 ? 1 : BX + 6;
        fN = k == 0 ? F_N1X : F_N2X;
        fNy = k == 0 ? F_N1Y : F_N2Y;
        fXT = k == 0 ? F_XT1 : F_XT2;
    }
    __device__ __forceinline__ int base(int line) const {
        return k == 0 ? (DIM == 2 ? (3 + line) * (BX + 6) : 0) : 3 + line;
    }
};

// ---- C: pair flux P_m(q) = F(U_q, U_{q+m}), q = 3-m .. LB+2, item t of direction d; stored at
// PB[c * ps + out]
template <int DIM, int BX, int BY>
__device__ __forceinline__ void pair_item(const double* S, int NB, const DirGeo<DIM, BX, BY>& d, int t, const Gas& G,
                                          double* PB, int ps, int out) {
    const int line = t / d.per_line, kk = t % d.per_line;
    int m, q;
    if (kk < d.LB + 1) { m = 1; q = 2 + kk; }
    else if (kk < 2 * d.LB + 3) { m = 2; q = 1 + (kk - d.LB - 1); }
    else { m = 3; q = kk - 2 * d.LB - 3; }
    const int l = d.base(line) + q * d.step, r = l + m * d.step;
    const double nx = 0.5 * (S[d.fN * NB + l] + S[d.fN * NB + r]);
    const double ny = 0.5 * (S[d.fNy * NB + l] + S[d.fNy * NB + r]);
    const double xt = 0.5 * (S[d.fXT * NB + l] + S[d.fXT * NB + r]);
    double f[DIM + 2];
    pair_flux<DIM>(S, NB, l, r, nx, ny, xt, G, f);
#pragma unroll
    for (int c = 0; c < DIM + 2; ++c) PB[c * ps + out] = f[c];
}

// ---- D: face flux at q+1/2, q = 2 .. LB+2 (box coordinates), item t of direction d: the 6th-order
// combination of the direction's pairs (which start at PB[c * ps + poff]) plus the dissipation;
// stored at FB[c * fs + out]
template <int DIM, int BX, int BY>
__device__ __forceinline__ void face_item(const double* S, int NB, const DirGeo<DIM, BX, BY>& d, int t,
                                          const StageParams& P, const double* PB, int ps, int poff, double* FB,
                                          int fs, int out) {
    constexpr int NC = DIM + 2;
    const int line = t / (d.LB + 1), f = t % (d.LB + 1);
    const int q = 2 + f;
    const int pbase = poff + line * d.per_line;
    double F[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) F[c] = 0.0;
    double FJ = 0.0;
    const int base = d.base(line);
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
        const int off = m == 1 ? 0 : (m == 2 ? d.LB + 1 : 2 * d.LB + 3);
        const double al = ec_alpha(m);
        for (int s = 0; s < m; ++s) {
            const int qq = q - s;                       // left node of the pair
            const int pi = pbase + off + (qq - (3 - m));
#pragma unroll
            for (int c = 0; c < NC; ++c) F[c] += al * PB[c * ps + pi];
            FJ += al * 0.5 * (S[d.fXT * NB + base + qq * d.step] + S[d.fXT * NB + base + (qq + m) * d.step]);
        }
    }
    if (P.diss) {
        const int l = base + q * d.step;
        const double nx = 0.5 * (S[d.fN * NB + l] + S[d.fN * NB + l + d.step]);
        const double ny = 0.5 * (S[d.fNy * NB + l] + S[d.fNy * NB + l + d.step]);
        const double xtf = 0.5 * (S[d.fXT * NB + l] + S[d.fXT * NB + l + d.step]);
        double dd[NC];
        face_dissipation<DIM>(S, NB, l, d.step, nx, ny, xtf, P.gas, P.weno, dd, P.status, 0);
#pragma unroll
        for (int c = 0; c < NC; ++c) F[c] += dd[c];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) FB[c * fs + out] = F[c];
    FB[NC * fs + out] = FJ;
}

template <int DIM, int BX, int BY, int NT>
__global__ void __launch_bounds__(NT, 1)
stage_kernel_fp64(StageParams P) {
    using TL = Tile<DIM, BX, BY, NT>;
    constexpr int GX = TL::GX, NB = TL::NB, NC = TL::NC;
    extern __shared__ double smem[];
    double* S = smem;                                   // F_COUNT * NB
    double* PB = smem + F_COUNT * NB;                   // pair buffer (also the coordinates)
    double* FB = PB + TL::PAIR_DOUBLES;                 // face buffer (NC + 1) * FS
    const int tid = threadIdx.x;
    const int ntx = (P.n1 + BX - 1) / BX;
    const int i0 = (blockIdx.x % ntx) * BX;
    const int j0 = DIM == 2 ? (blockIdx.x / ntx) * BY : 0;
    const double dt = P.dt_dev ? *P.dt_dev : P.dt_host;
    if (P.mode == 0 && dt == 0.0) return;               // finished run: leave the state untouched
    const double cdt = P.cst * dt;
    const Gas& G = P.gas;

    // ---- A: coordinates of the whole box, node data of the cross-shaped halo
    double* XS = PB;            // DIM * NB
    double* XD = PB + 2 * NB;   // DIM * NB
    for (int b = tid; b < NB; b += TL::THREADS) {
        const int ii = b % GX, jj = b / GX;
        const int gi = i0 - 3 + ii, gj = j0 - 3 + jj;
        double xs[2], xd[2];
        stage_coords<DIM>(P, gi, DIM == 2 ? gj : 0, cdt, xs, xd);
        XS[b] = xs[0];
        XD[b] = xd[0];
        if (DIM == 2) {
            XS[NB + b] = xs[1];
            XD[NB + b] = xd[1];
        }
        const bool in_x = ii >= 3 && ii < 3 + BX;
        const bool in_y = DIM == 1 || (jj >= 3 && jj < 3 + BY);
        if (in_x || in_y) load_node<DIM>(S, NB, b, P, gi, gj);
    }
    __syncthreads();

    // ---- B: metrics of the stage mesh (eq. SCLCoeff degenerate to 2D, eq. VCLCoeff)
    for (int b = tid; b < NB; b += TL::THREADS) {
        const int ii = b % GX, jj = b / GX;
        if (DIM == 1) {
            S[F_N1X * NB + b] = 1.0;
            S[F_N1Y * NB + b] = 0.0;
            S[F_XT1 * NB + b] = -XD[b];
        } else {
            if (jj >= 3 && jj < 3 + BY) {          // xi_1 lines: J dxi_1/dx = (d2 y, -d2 x)/dxi_2
                double dy = 0.0, dx = 0.0;
#pragma unroll
                for (int m = 1; m <= 3; ++m) {
                    const double h = 0.5 * ec_alpha(m);
                    dx += h * (XS[b + m * GX] - XS[b - m * GX]);
                    dy += h * (XS[NB + b + m * GX] - XS[NB + b - m * GX]);
                }
                const double nx = dy * P.inv_dxi[1], ny = -dx * P.inv_dxi[1];
                S[F_N1X * NB + b] = nx;
                S[F_N1Y * NB + b] = ny;
                S[F_XT1 * NB + b] = -(XD[b] * nx + XD[NB + b] * ny);
            }
            if (ii >= 3 && ii < 3 + BX) {          // xi_2 lines: J dxi_2/dx = (-d1 y, d1 x)/dxi_1
                double dy = 0.0, dx = 0.0;
#pragma unroll
                for (int m = 1; m <= 3; ++m) {
                    const double h = 0.5 * ec_alpha(m);
                    dx += h * (XS[b + m] - XS[b - m]);
                    dy += h * (XS[NB + b + m] - XS[NB + b - m]);
                }
                const double nx = -dy * P.inv_dxi[0], ny = dx * P.inv_dxi[0];
                S[F_N2X * NB + b] = nx;
                S[F_N2Y * NB + b] = ny;
                S[F_XT2 * NB + b] = -(XD[b] * nx + XD[NB + b] * ny);
            }
        }
    }
    __syncthreads();

    double acc[NC + 1];
#pragma unroll
    for (int c = 0; c <= NC; ++c) acc[c] = 0.0;
    const int tx = tid % BX, ty = tid / BX;

    // ---- C, D, E: pairs, faces and the divergence at the interior node (tx, ty)
    if constexpr (TL::JOINT) {
        // a warp may hold items of both directions: the direction is data (one code path), not a branch
        for (int t = tid; t < TL::NP1 + TL::NP2; t += TL::THREADS) {
            const bool two = t >= TL::NP1;
            pair_item<DIM, BX, BY>(S, NB, DirGeo<DIM, BX, BY>(two ? 1 : 0), two ? t - TL::NP1 : t, G, PB, TL::PS, t);
        }
        __syncthreads();
        for (int t = tid; t < TL::NF1 + TL::NF2; t += TL::THREADS) {
            const bool two = t >= TL::NF1;
            face_item<DIM, BX, BY>(S, NB, DirGeo<DIM, BX, BY>(two ? 1 : 0), two ? t - TL::NF1 : t, P, PB, TL::PS,
                                   two ? TL::POFF2 : 0, FB, TL::FS, t);
        }
        __syncthreads();
        if (tid < BX * BY) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int LB = k == 0 ? BX : BY;
                const int fm = (k == 0 ? 0 : TL::FOFF2) + (k == 0 ? ty : tx) * (LB + 1) + (k == 0 ? tx : ty);
                const double inv = P.inv_dxi[k];
#pragma unroll
                for (int c = 0; c <= NC; ++c) acc[c] -= (FB[c * TL::FS + fm + 1] - FB[c * TL::FS + fm]) * inv;
            }
        }
    } else {
#pragma unroll 1
        for (int k = 0; k < DIM; ++k) {
            const DirGeo<DIM, BX, BY> d(k);
            for (int t = tid; t < d.nlines * d.per_line; t += TL::THREADS)
                pair_item<DIM, BX, BY>(S, NB, d, t, G, PB, TL::PS, t);
            __syncthreads();
            for (int t = tid; t < d.nlines * (d.LB + 1); t += TL::THREADS)
                face_item<DIM, BX, BY>(S, NB, d, t, P, PB, TL::PS, 0, FB, TL::FS, t);
            __syncthreads();
            if (tid < BX * (DIM == 2 ? BY : 1)) {
                const int line = k == 0 ? ty : tx;
                const int pos = k == 0 ? tx : ty;
                const int fm = line * (d.LB + 1) + pos;           // face pos - 1/2
                const double inv = P.inv_dxi[k];
#pragma unroll
                for (int c = 0; c <= NC; ++c) acc[c] -= (FB[c * TL::FS + fm + 1] - FB[c * TL::FS + fm]) * inv;
            }
            __syncthreads();
        }
    }

    // ---- F: Shu-Osher combination (or the bare right-hand side)
    const int gi = i0 + tx, gj = j0 + ty;
    if (tid < BX * (DIM == 2 ? BY : 1) && gi < P.n1 && (DIM == 1 || gj < P.n2)) {
        const size_t N = size_t(P.n1) * P.n2;
        const size_t idx = size_t(DIM == 2 ? gj : 0) * P.n1 + gi;
        if (P.mode == 1) {
#pragma unroll
            for (int c = 0; c < NC; ++c) P.JUo[c * N + idx] = acc[c];
            P.Jo[idx] = acc[NC];
        } else {
            // all operands loaded before the first store (a store may alias a later load as far as the compiler
            // knows, which would serialise one round trip per component)
            double un[NC], us[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                un[c] = P.JUn[c * N + idx];
                us[c] = P.JUs[c * N + idx];
            }
            const double Jn = P.Jn[idx];
            const double Js = P.Js[idx];
#pragma unroll
            for (int c = 0; c < NC; ++c) P.JUo[c * N + idx] = P.ca * un[c] + P.cb * (us[c] + dt * acc[c]);
            const double Jnew = P.ca * Jn + P.cb * (Js + dt * acc[NC]);
            P.Jo[idx] = Jnew;
            if (!(Jnew > 0.0)) raise_error(P.status, ES_ERR_MESH, int(idx));
        }
    }
}

// ----------------------------------------------------------------- launch
template <int DIM, int BX, int BY, int NT>
static cudaError_t prepare_tile() {
    return cudaFuncSetAttribute(stage_kernel_fp64<DIM, BX, BY, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(Tile<DIM, BX, BY, NT>::SMEM));
}

template <int DIM, int BX, int BY, int NT>
static cudaError_t launch_tile(const StageParams& P, cudaStream_t s) {
    using TL = Tile<DIM, BX, BY, NT>;
    const int ntx = (P.n1 + BX - 1) / BX;
    const int nty = DIM == 2 ? (P.n2 + BY - 1) / BY : 1;
    stage_kernel_fp64<DIM, BX, BY, NT><<<ntx * nty, NT, TL::SMEM, s>>>(P);
    return cudaGetLastError();
}

// 2D shapes: 32 x 8 nodes with 288 threads (= the 32 x 9 faces of xi_2), 25 x 11 with 384
// (25 x 12 = 300 faces; 8 x 19 = 152 tiles cover 200 x 200 in one wave on 152 SMs), 16 x 16
// with 288 (272 faces), 32 x 12 with 416 (416 faces; less halo per node), 20 x 10 with 224.  1D: 254 nodes, 256 threads (255 faces, 768 pairs = three passes).
cudaError_t stage_prepare_fp64(int dim) {
    if (dim == 1) return prepare_tile<1, 254, 1, 256>();
    cudaError_t e = prepare_tile<2, 32, 8, 288>();
    if (e == cudaSuccess) e = prepare_tile<2, 25, 11, 384>();
    if (e == cudaSuccess) e = prepare_tile<2, 16, 16, 288>();
    if (e == cudaSuccess) e = prepare_tile<2, 32, 12, 416>();
    if (e == cudaSuccess) e = prepare_tile<2, 20, 10, 224>();
    return e;
}

cudaError_t launch_stage_fp64(const StageParams& P, cudaStream_t s) {
    if (P.dim == 1) return launch_tile<1, 254, 1, 256>(P, s);
    switch (P.tile) {
        case 1: return launch_tile<2, 25, 11, 384>(P, s);
        case 2: return launch_tile<2, 16, 16, 288>(P, s);
        case 3: return launch_tile<2, 32, 12, 416>(P, s);
        case 4: return launch_tile<2, 20, 10, 224>(P, s);
        default: return launch_tile<2, 32, 8, 288>(P, s);
    }
}

void stage_tile_shape(bool mixed, int k, int* bx, int* by, int* nt) {
    static const int fp64[STAGE_NTILES][3] = {{32, 8, 288}, {25, 11, 384}, {16, 16, 288}, {32, 12, 416},
                                              {20, 10, 224}};
    static const int f32[STAGE_NTILES][3] = {{32, 8, 288}, {25, 6, 192}, {20, 8, 192}, {32, 16, 544}, {16, 8, 160}};
    const int(*t)[3] = mixed ? f32 : fp64;
    *bx = t[k][0];
    *by = t[k][1];
    *nt = t[k][2];
}

}  // namespace es
