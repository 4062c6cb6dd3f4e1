// es_3d.cu -- the ES operator, SSP-RK3 stage and mesh redistribution in three dimensions (FP64).
//
// A 3D tile with a 3-node halo in every direction holds (BX+6)(BY+6)(BZ+6) nodes: in FP64
// that is several times the shared memory of an SM for any useful tile, so the 3D path is
// split by direction instead:
//   k3_coords   stage coordinates x^n + c dt xdot on the mesh extended by 3 ghosts (Sec. 3.2)
//   k3_deriv    delta_l[x_p] there (the inner differences of eq. SCLCoeff)
//   k3_metric   J dxi_k/dx_j = (delta_m[delta_l[x_p] x_q] - delta_l[delta_m[x_p] x_q])/(dxi_l dxi_m)
//               for (k, l, m), (j, p, q) cyclic (eq. SCLCoeff), on each direction's nodes plus
//               3 ghosts along xi_k
//   k3_nodes    primitive state, logarithms and entropy variables of every node, once
//   k3_dir<K>   per xi_K: pencils of LB nodes x W lines staged in shared memory; pair fluxes
//               (eq. ECfluxMM), the 6th-order combination (eq. ECFlux_curv_2p, GCL_flux), the ES
//               dissipation with the theta/phi rotation (eq. HOstable, Sec. 3.3) and the
//               divergence, accumulated over the directions; the last direction applies the
//               Shu-Osher combination.
// The mesh redistribution (Sec. 4) uses 3D monitor, filter, Jacobi and limiter kernels and
// shares the elementwise kernels of the 1D/2D path.
#include <cuda_runtime.h>

#include "es_3d.h"
#include "es_3d_grid.cuh"
#include "es_device.cuh"
#include "es_internal.h"

namespace es {

// node fields of the 3D path (global planes and shared-memory slots)
enum Field3 {
    G_RHO, G_V1, G_V2, G_V3, G_T, G_IT, G_OM, G_IOM, G_G, G_RT, G_VT1, G_VT2, G_VT3, G_V2T,
    G_RV1, G_RV2, G_RV3, G_LNR, G_LNOM, G_LNT, G_RP, G_LNRP, G_W0,
    F3_COUNT,
    G_NX = F3_COUNT, G_NY, G_NZ, G_XT,     // metrics of the direction (shared memory only)
    S3_COUNT
};

// field at a possibly-ghost node, ghosts by copy / wrap (monitor and filter)
__device__ __forceinline__ double field3(const Grid3& g, const double* f, int i1, int i2, int i3) {
    return f[idx3(g, state_index(i1, g.n[0], g.bc[0]), state_index(i2, g.n[1], g.bc[1]),
                  state_index(i3, g.n[2], g.bc[2]))];
}

// stride of direction k in a [n3][n2][n1] field
__device__ __forceinline__ size_t stride3(const Grid3& g, int k) {
    return k == 0 ? 1 : (k == 1 ? size_t(g.n[0]) : size_t(g.n[0]) * g.n[1]);
}

// index of the node at offset s (|s| = 1) along direction k from in-mesh node id (position i_k),
// ghosts by copy / wrap: the neighbour can leave the mesh along k only
__device__ __forceinline__ size_t nb_index(const Grid3& g, size_t id, int ik, int k, int s) {
    const int j = state_index(ik + s, g.n[k], g.bc[k]);
    return id + (long long)(j - ik) * (long long)stride3(g, k);
}

// coordinate component `comp` of that neighbour: wrap with the period shift, or odd reflection
// about the boundary node (2 x_b - x_{b -+ 1}), the one-direction case of the ghost rule
__device__ __forceinline__ double nb_coord(const Grid3& g, const double* f, size_t id, int ik, int k, int s,
                                           int comp) {
    const int n = g.n[k];
    const int j = ik + s;
    const long long st = (long long)stride3(g, k);
    if (j >= 0 && j < n) return f[id + (long long)s * st];
    if (g.bc[k] == ES_BC_PERIODIC) {
        const int r = j < 0 ? j + n : j - n;
        double v = f[id + (long long)(r - ik) * st];
        if (comp == k) v += (j < 0 ? -1.0 : 1.0) * g.period[k];
        return v;
    }
    const int b = j < 0 ? 0 : n - 1, m = j < 0 ? 1 : n - 2;
    if (comp != k && end_mirrored(g.bc[k], j < 0)) return f[id + (long long)(m - ik) * st];
    return 2.0 * f[id + (long long)(b - ik) * st] - f[id + (long long)(m - ik) * st];
}

__device__ __forceinline__ double block_max(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}

__device__ __forceinline__ double block_min(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = threadIdx.x < nw ? sh[threadIdx.x] : 1e300;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}

// ================================================================ metrics
// stage coordinates on the extended grid
__global__ void k3_coords(Grid3 g, const double* xn, const double* xdot, double cst, const double* dt_dev,
                          double dt_host, double* XE) {
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    const int E1 = g.n[0] + 6, E2 = g.n[1] + 6, E3 = g.n[2] + 6;
    const size_t NE = size_t(E1) * E2 * E3;
    const double cdt = cst * (dt_dev ? *dt_dev : dt_host);
    for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < NE; e += size_t(gridDim.x) * blockDim.x) {
        const int e1 = int(e % E1), e2 = int((e / E1) % E2), e3 = int(e / (size_t(E1) * E2));
        const int i1 = e1 - 3, i2 = e2 - 3, i3 = e3 - 3;
        if (inside3(g, i1, i2, i3, 0)) {
            const size_t id = idx3(g, i1, i2, i3);
            for (int c = 0; c < 3; ++c) XE[c * NE + e] = xdot ? xn[c * N + id] + cdt * xdot[c * N + id] : xn[c * N + id];
            continue;
        }
        for (int c = 0; c < 3; ++c)
            XE[c * NE + e] = ghost_value3(g, xn + c * N, xdot ? xdot + c * N : nullptr, cdt, i1, i2, i3, c);
    }
}

// The products of eq. SCLCoeff's cross form, once per node: D[3 l + j] = delta_l[x_p] x_q with
// p = (j + 1) % 3, q = (j + 2) % 3 (delta_l undivided; 0 where the xi_l index is not interior).
// Each is differenced by two directions' metrics, which therefore read the same rounded value.
__global__ void k3_deriv(Grid3 g, const double* XE, double* D) {
    const int E1 = g.n[0] + 6, E2 = g.n[1] + 6, E3 = g.n[2] + 6;
    const size_t NE = size_t(E1) * E2 * E3;
    const size_t st[3] = {1, size_t(E1), size_t(E1) * E2};
    for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < NE; e += size_t(gridDim.x) * blockDim.x) {
        const int ee[3] = {int(e % E1), int((e / E1) % E2), int(e / (size_t(E1) * E2))};
        const double x[3] = {XE[e], XE[NE + e], XE[2 * NE + e]};
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const bool ok = ee[l] >= 3 && ee[l] < g.n[l] + 3;
            double dl[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                double s = 0.0;
                if (ok) {
#pragma unroll
                    for (int m = 1; m <= 3; ++m)
                        s += 0.5 * ec_alpha(m) * (XE[p * NE + e + m * st[l]] - XE[p * NE + e - m * st[l]]);
                }
                dl[p] = s;
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) D[(3 * l + j) * NE + e] = dl[(j + 1) % 3] * x[(j + 2) % 3];
        }
    }
}

// J dxi_k/dx_j on direction k's grid (n_k + 6 nodes along xi_k, interior across); the direction is a template
// parameter (no run-time indexing of the grid's arrays)
template <int k>
__global__ void k3_metric(Grid3 g, const double* D, double* NKo) {
    const int E1 = g.n[0] + 6, E2 = g.n[1] + 6;
    const size_t NE = size_t(E1) * E2 * (g.n[2] + 6);
    int m1 = g.n[0], m2 = g.n[1], m3 = g.n[2];
    if (k == 0) m1 += 6;
    else if (k == 1) m2 += 6;
    else m3 += 6;
    const size_t M = size_t(m1) * m2 * m3;
    const int l = (k + 1) % 3, m = (k + 2) % 3;
    const double scale = g.inv_dxi[l] * g.inv_dxi[m];
    const size_t stl = l == 0 ? 1 : (l == 1 ? size_t(E1) : size_t(E1) * E2);
    const size_t stm = m == 0 ? 1 : (m == 1 ? size_t(E1) : size_t(E1) * E2);
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < M; t += size_t(gridDim.x) * blockDim.x) {
        const int a1 = int(t % m1), a2 = int((t / m1) % m2), a3 = int(t / (size_t(m1) * m2));
        // extended-grid position: the metric grid already carries the 3 ghosts along xi_k
        const size_t e = eidx(g, a1 + (k == 0 ? 0 : 3), a2 + (k == 1 ? 0 : 3), a3 + (k == 2 ? 0 : 3));
        for (int j = 0; j < 3; ++j) {
            const double* Pl = D + (3 * l + j) * NE;      // delta_l[x_p] x_q
            const double* Pm = D + (3 * m + j) * NE;      // delta_m[x_p] x_q
            double A = 0.0, B = 0.0;
#pragma unroll
            for (int a = 1; a <= 3; ++a) {
                const double h = 0.5 * ec_alpha(a);
                const size_t sm = a * stm, sl = a * stl;
                A += h * (Pl[e + sm] - Pl[e - sm]);
                B += h * (Pm[e + sl] - Pm[e - sl]);
            }
            NKo[j * M + t] = (A - B) * scale;
        }
    }
}

// ================================================================ node fields
__global__ void k3_nodes(Grid3 g, Gas G, const double* JU, const double* J, double* NF, DevStatus* st) {
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    for (size_t id = blockIdx.x * size_t(blockDim.x) + threadIdx.x; id < N; id += size_t(gridDim.x) * blockDim.x) {
        const double iJ = rcp_nr(J[id]);
        const double rho = JU[id] * iJ;
        const double m1 = JU[N + id] * iJ, m2 = JU[2 * N + id] * iJ, m3 = JU[3 * N + id] * iJ;
        const double E = JU[4 * N + id] * iJ;
        const double irho = rcp_nr(rho);
        const double v1 = m1 * irho, v2 = m2 * irho, v3 = m3 * irho;
        const double ke = 0.5 * (v1 * v1 + v2 * v2 + v3 * v3);
        const double T = (E * irho - ke + G.a * rho) * G.icv;
        const double om = 1.0 - G.b * rho;
        const double iom = rcp_nr(om);
        const double p = rho * G.R * T * iom - G.a * rho * rho;
        const double iT = rcp_nr(T);
        if (!(rho > 0.0) || !(om > 0.0) || !(T > 0.0) || !(p > 0.0)) raise_error(st, ES_ERR_INADMISSIBLE, int(id));
        const double lnr = log(rho);
        const double lnom = G.b > 0.0 ? log(om) : 0.0;
        const double lnT = log(T);
        const double lnp = log(p);
        NF[G_RHO * N + id] = rho;
        NF[G_V1 * N + id] = v1;
        NF[G_V2 * N + id] = v2;
        NF[G_V3 * N + id] = v3;
        NF[G_T * N + id] = T;
        NF[G_IT * N + id] = iT;
        NF[G_OM * N + id] = om;
        NF[G_IOM * N + id] = iom;
        NF[G_G * N + id] = G.R * iom - G.a * rho * iT;
        NF[G_RT * N + id] = rho * iT;
        NF[G_VT1 * N + id] = v1 * iT;
        NF[G_VT2 * N + id] = v2 * iT;
        NF[G_VT3 * N + id] = v3 * iT;
        NF[G_V2T * N + id] = 2.0 * ke * iT;
        NF[G_RV1 * N + id] = m1;
        NF[G_RV2 * N + id] = m2;
        NF[G_RV3 * N + id] = m3;
        NF[G_LNR * N + id] = lnr;
        NF[G_LNOM * N + id] = lnom;
        NF[G_LNT * N + id] = lnT;
        NF[G_RP * N + id] = div_nr(rho, p);
        NF[G_LNRP * N + id] = lnr - lnp;
        // entropy variables V = ((e + p/rho)/T - s - |v|^2/(2T), v/T, -1/T); V_1..3 = VT, V_4 = -IT
        const double s = G.cv * lnT + G.R * (lnom - lnr);
        NF[G_W0 * N + id] = G.cv - s - 2.0 * G.a * rho * iT + G.R * iom - ke * iT;
    }
}

// ================================================================ direction flux
// two-point EC flux of Sec. 3.1 contracted with the face-averaged metrics (n, J xi_t)
__device__ __forceinline__ void pair_flux3(const double* S, int NB, int l, int r, double nx, double ny, double nz,
                                           double xt, const Gas& G, double* out) {
    const double rl = S[G_RHO * NB + l], rr = S[G_RHO * NB + r];
    const double Tl = S[G_T * NB + l], Tr = S[G_T * NB + r];
    const double rho_m = 0.5 * (rl + rr);
    const double T_m = 0.5 * (Tl + Tr);
    const double iT_m = 0.5 * (S[G_IT * NB + l] + S[G_IT * NB + r]);
    const double ilr = inv_log_mean(rl, rr, S[G_LNR * NB + l], S[G_LNR * NB + r]);
    const double ilT = inv_log_mean(Tl, Tr, S[G_LNT * NB + l], S[G_LNT * NB + r]);
    const double Pinv = S[G_IOM * NB + l] * S[G_IOM * NB + r];
    const double iTa = rcp_nr(T_m);
    const double coef = G.R * G.b * Pinv - G.a * iTa;
    double D = G.R * ilr + coef - G.a * iTa;
    if (G.b > 0.0)
        D += G.R * G.b * inv_log_mean(S[G_OM * NB + l], S[G_OM * NB + r], S[G_LNOM * NB + l], S[G_LNOM * NB + r]);
    const double iD = rcp_nr(D);
    const double g_m = 0.5 * (S[G_G * NB + l] + S[G_G * NB + r]);
    const double rT_m = 0.5 * (S[G_RT * NB + l] + S[G_RT * NB + r]);
    const double v2T_m = 0.5 * (S[G_V2T * NB + l] + S[G_V2T * NB + r]);
    double vm[3], vT[3], rv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        vm[c] = 0.5 * (S[(G_V1 + c) * NB + l] + S[(G_V1 + c) * NB + r]);
        vT[c] = 0.5 * (S[(G_VT1 + c) * NB + l] + S[(G_VT1 + c) * NB + r]);
        rv[c] = 0.5 * (S[(G_RV1 + c) * NB + l] + S[(G_RV1 + c) * NB + r]);
    }
    const double U1 = (rho_m * coef + g_m) * iD;
    const double F11 = (rv[0] * coef + g_m * vm[0]) * iD;
    const double F21 = (rv[1] * coef + g_m * vm[1]) * iD;
    const double F31 = (rv[2] * coef + g_m * vm[2]) * iD;
    const double P = rho_m * T_m * g_m;
    const double B0 = 0.5 * v2T_m - G.cv * T_m * ilT + 2.0 * G.a * rT_m;
    const double Q1 = xt * U1 + nx * F11 + ny * F21 + nz * F31;
    const double sv = vT[0] * vm[0] + vT[1] * vm[1] + vT[2] * vm[2];
    out[0] = Q1;
    out[1] = vm[0] * Q1 + nx * P;
    out[2] = vm[1] * Q1 + ny * P;
    out[3] = vm[2] * Q1 + nz * P;
    out[4] = div_nr(G.a * rT_m * (xt * rho_m + nx * rv[0] + ny * rv[1] + nz * rv[2]) + (sv - B0) * Q1 +
                        P * (nx * vT[0] + ny * vT[1] + nz * vT[2]),
                    iT_m);
}

// -1/2 Lambda T^{-1} R Y [[W]]^WENO at the face between pencil nodes l and l+1 (Sec. 3.3,
// eq. HOstable) with the 3D rotation: theta = atan2(n_2, n_1) (0 when |(n_1, n_2)| <= 1e-12 |n|, the
// rounding of metrics that vanish exactly),
// phi = atan2(n_3, sqrt(n_1^2 + n_2^2)), so the rows of T's momentum block are
// e_n = n/L, e_t1 = (-sin theta, cos theta, 0), e_t2 = (-sin phi cos theta, -sin phi sin theta, cos phi);
// R's tangential columns are (0, 0, 1, 0, v_t1) and (0, 0, 0, 1, v_t2), scaled by sqrt(rho T).
__device__ __forceinline__ void face_dissipation3(const double* S, int NB, int l, double nx, double ny, double nz,
                                                  double xtf, const Gas& G, const Weno& Wc, double* out,
                                                  DevStatus* st) {
    const int r = l + 1;
    const double ilr = inv_log_mean(S[G_RHO * NB + l], S[G_RHO * NB + r], S[G_LNR * NB + l], S[G_LNR * NB + r]);
    const double rho = rcp_nr(ilr);
    const double ilrp = inv_log_mean(S[G_RP * NB + l], S[G_RP * NB + r], S[G_LNRP * NB + l], S[G_LNRP * NB + r]);
    const double p = rho * ilrp;
    const double om = 1.0 - G.b * rho;
    const double T = (p + G.a * rho * rho) * om * ilr * G.iR;
    const double iom = rcp_nr(om);
    const double c2 = (1.0 + G.delta) * G.R * T * iom * iom - 2.0 * G.a * rho;
    const double dcrit = G.R * T - 2.0 * G.a * rho * om * om;
    if (!(c2 > 0.0) || !(dcrit > 0.0) || !(om > 0.0)) raise_error(st, ES_ERR_INADMISSIBLE, 0);
    const double c = sqrt(c2);
    const double vm1 = 0.5 * (S[G_V1 * NB + l] + S[G_V1 * NB + r]);
    const double vm2 = 0.5 * (S[G_V2 * NB + l] + S[G_V2 * NB + r]);
    const double vm3 = 0.5 * (S[G_V3 * NB + l] + S[G_V3 * NB + r]);
    const double L = sqrt(nx * nx + ny * ny + nz * nz);
    const double r12 = sqrt(nx * nx + ny * ny);
    double ct = 1.0, sn = 0.0;
    if (r12 > 1e-12 * L) {
        const double ir = rcp_nr(r12);
        ct = nx * ir;
        sn = ny * ir;
    }
    const double iL = rcp_nr(L);
    const double cp = r12 * iL, sp = nz * iL;
    const double en[3] = {cp * ct, cp * sn, sp};
    const double et1[3] = {-sn, ct, 0.0};
    const double et2[3] = {-sp * ct, -sp * sn, cp};
    const double vn = en[0] * vm1 + en[1] * vm2 + en[2] * vm3;
    const double vt1 = et1[0] * vm1 + et1[1] * vm2;
    const double vt2 = et2[0] * vm1 + et2[1] * vm2 + et2[2] * vm3;
    const double E = rho * (G.cv * T - G.a * rho) + 0.5 * rho * (vn * vn + vt1 * vt1 + vt2 * vt2);
    const double H = (E + p) * ilr;
    const double mid = H - c2 * om * G.idelta;
    const double ic2 = rcp_nr(c2);
    const double sA = sqrt(0.5 * rho * T * ic2);
    const double sE = sqrt(div_nr(G.R * G.delta * rho * T * T * ic2, dcrit));
    const double sT = sqrt(rho * T);
    const double Lam = fabs(xtf + L * vn) + L * c;
    const double Hm = H - vn * c, Hp = H + vn * c;

    // W = R^T (T V) at nodes l-2 .. l+3
    double W[6][5];
    double aTV[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        const int q = l + (o - 2);
        const double V0 = S[G_W0 * NB + q];
        const double a1 = S[G_VT1 * NB + q], a2 = S[G_VT2 * NB + q], a3 = S[G_VT3 * NB + q];
        const double V4 = -S[G_IT * NB + q];
        const double V1 = en[0] * a1 + en[1] * a2 + en[2] * a3;
        const double V2 = et1[0] * a1 + et1[1] * a2;
        const double V3 = et2[0] * a1 + et2[1] * a2 + et2[2] * a3;
        const double base = V0 + vt1 * V2 + vt2 * V3;
        W[o][0] = sA * (base + (vn - c) * V1 + Hm * V4);
        W[o][1] = sE * (base + vn * V1 + mid * V4);
        W[o][2] = sT * (V2 + vt1 * V4);
        W[o][3] = sT * (V3 + vt2 * V4);
        W[o][4] = sA * (base + (vn + c) * V1 + Hp * V4);
        if (o == 2 || o == 3) {
            aTV[0] += fabs(V0);
            aTV[1] += fabs(V1);
            aTV[2] += fabs(V2);
            aTV[3] += fabs(V3);
            aTV[4] += fabs(V4);
        }
    }
    const double avt1 = fabs(vt1), avt2 = fabs(vt2);
    const double common = aTV[0] + avt1 * aTV[2] + avt2 * aTV[3];
    double scl[5];
    scl[0] = sA * (common + fabs(vn - c) * aTV[1] + fabs(Hm) * aTV[4]);
    scl[1] = sE * (common + fabs(vn) * aTV[1] + fabs(mid) * aTV[4]);
    // tangential waves: round-off in a velocity follows the flow's velocity scale |v_t| + c
    scl[2] = sT * (aTV[2] + (avt1 + c) * aTV[4]);
    scl[3] = sT * (aTV[3] + (avt2 + c) * aTV[4]);
    scl[4] = sA * (common + fabs(vn + c) * aTV[1] + fabs(Hp) * aTV[4]);
    double y[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const double wmin = mr_weno5(W[0][m], W[1][m], W[2][m], W[3][m], W[4][m], Wc);
        const double wplu = mr_weno5(W[5][m], W[4][m], W[3][m], W[2][m], W[1][m], Wc);
        const double jw = wplu - wmin;
        double j = W[3][m] - W[2][m];
        if (fabs(j) <= Wc.sign_tol * scl[m]) j = 0.0;
        const bool keep = (jw > 0.0 && j > 0.0) || (jw < 0.0 && j < 0.0);
        y[m] = keep ? jw : 0.0;
    }
    const double h = -0.5 * Lam;
    const double y0 = sA * y[0], y1 = sE * y[1], y2 = sT * y[2], y3 = sT * y[3], y4 = sA * y[4];
    const double i0 = y0 + y1 + y4;
    const double i1 = (vn - c) * y0 + vn * y1 + (vn + c) * y4;
    const double i2 = vt1 * i0 + y2;
    const double i3 = vt2 * i0 + y3;
    const double i4 = Hm * y0 + mid * y1 + vt1 * y2 + vt2 * y3 + Hp * y4;
    out[0] = h * i0;
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) out[1 + c3] = h * (en[c3] * i1 + et1[c3] * i2 + et2[c3] * i3);
    out[4] = h * i4;
}

struct Dir3Params {
    Grid3 g;
    Gas gas;
    Weno weno;
    int diss;
    const double* NF;         // node fields [F3_COUNT][N]
    const double* NK;         // metrics of this direction [3][M]
    const double* xdot;       // nullable
    double* RH;               // accumulated right-hand sides [6][N]
    int first, last;
    int mode;                 // last direction: 0 RK combination, 1 right-hand sides out
    double ca, cb;
    double dt_host;
    const double* dt_dev;
    const double *JUn, *Jn, *JUs, *Js;
    double *JUo, *Jo;
    DevStatus* status;
};

template <int LB, int W>
struct Pencil {
    static constexpr int LS = (LB + 6) | 1;             // node stride of a line (odd: no bank conflicts)
    static constexpr int NB = W * LS;
    static constexpr int PL = 3 * LB + 6;               // pairs per line
    static constexpr int NP = W * PL;
    static constexpr int NF = W * (LB + 1);             // faces
    static constexpr size_t SMEM = sizeof(double) * (size_t(S3_COUNT) * NB + 5 * NP + 6 * NF);
};

template <int K, int LB, int W, int NT>
__global__ void __launch_bounds__(NT, W >= 16 ? 1 : (NT <= 96 ? 3 : 2)) k3_dir(Dir3Params P) {
    using PC = Pencil<LB, W>;
    constexpr int LS = PC::LS, NB = PC::NB, NP = PC::NP, NFc = PC::NF;
    extern __shared__ double smem[];
    double* S = smem;
    double* PB = S + S3_COUNT * NB;
    double* FB = PB + 5 * NP;
    const Grid3& g = P.g;
    const int tid = threadIdx.x;
    const int nk = g.n[K];
    // transverse indices: A (W consecutive lines) and B
    const int nA = K == 0 ? g.n[1] : g.n[0];
    const int nB = K == 2 ? g.n[1] : g.n[2];
    const int nseg = (nk + LB - 1) / LB;
    const int ngA = (nA + W - 1) / W;
    const int seg = blockIdx.x % nseg;
    const int grp = blockIdx.x / nseg;
    const int a0 = (grp % ngA) * W;
    const int b = grp / ngA;
    if (b >= nB) return;
    const int s0 = seg * LB;
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    const double dt = P.dt_dev ? *P.dt_dev : P.dt_host;
    if (P.mode == 0 && P.dt_dev && dt == 0.0) return;   // finished run: leave the state untouched
    const int M1 = g.n[0] + (K == 0 ? 6 : 0), M2 = g.n[1] + (K == 1 ? 6 : 0), M3 = g.n[2] + (K == 2 ? 6 : 0);
    const size_t M = size_t(M1) * M2 * M3;

    // ---- A: node fields and metrics of the pencils (3 ghosts along xi_K)
    for (int t = tid; t < W * (LB + 6); t += NT) {
        int line, q;
        if (K == 0) { line = t / (LB + 6); q = t % (LB + 6); }
        else { q = t / W; line = t % W; }
        int a = a0 + line;
        if (a > nA - 1) a = nA - 1;                          // ragged group: a valid line, not written
        const int s = s0 + q - 3;                            // along xi_K, possibly a ghost
        const int ss = state_index(s, nk, g.bc[K]);
        int i1, i2, i3, j1, j2, j3;
        if (K == 0) { i1 = ss; i2 = a; i3 = b; }
        else if (K == 1) { i1 = a; i2 = ss; i3 = b; }
        else { i1 = a; i2 = b; i3 = ss; }
        const size_t id = idx3(g, i1, i2, i3);
        const int bx = line * LS + q;
        double v[F3_COUNT];                                  // all loads in flight before the stores
#pragma unroll
        for (int f = 0; f < F3_COUNT; ++f) v[f] = P.NF[f * N + id];
#pragma unroll
        for (int f = 0; f < F3_COUNT; ++f) S[f * NB + bx] = v[f];
        if ((s < 0 || s >= nk) && end_mirrored(g.bc[K], s < 0)) {     // wall / symmetry ghost
            S[(G_V1 + K) * NB + bx] = -S[(G_V1 + K) * NB + bx];
            S[(G_VT1 + K) * NB + bx] = -S[(G_VT1 + K) * NB + bx];
            S[(G_RV1 + K) * NB + bx] = -S[(G_RV1 + K) * NB + bx];
        }
        // metrics: the metric grid holds s in [-3, n_K + 3); the tail of a ragged pencil is clamped
        int se = s + 3;
        se = se < 0 ? 0 : (se > nk + 5 ? nk + 5 : se);
        if (K == 0) { j1 = se; j2 = a; j3 = b; }
        else if (K == 1) { j1 = a; j2 = se; j3 = b; }
        else { j1 = a; j2 = b; j3 = se; }
        const size_t mi = (size_t(j3) * M2 + j2) * M1 + j1;
        const double nx = P.NK[mi], ny = P.NK[M + mi], nz = P.NK[2 * M + mi];
        S[G_NX * NB + bx] = nx;
        S[G_NY * NB + bx] = ny;
        S[G_NZ * NB + bx] = nz;
        double xt = 0.0;
        if (P.xdot) {
            // mesh velocity at the node: wrap, odd reflection, or at a wall / symmetry end the
            // mirror image (components along the plane mirrored, the normal one reflected)
            double xd[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const GhostTerms tk = ghost_terms(s, nk, g.bc[K], c != K);
                for (int u = 0; u < tk.nterm; ++u) {
                    int k1 = i1, k2 = i2, k3 = i3;
                    if (K == 0) k1 = tk.idx[u];
                    else if (K == 1) k2 = tk.idx[u];
                    else k3 = tk.idx[u];
                    xd[c] += tk.w[u] * P.xdot[c * N + idx3(g, k1, k2, k3)];
                }
            }
            xt = -(xd[0] * nx + xd[1] * ny + xd[2] * nz);
        }
        S[G_XT * NB + bx] = xt;
    }
    __syncthreads();

    // ---- C: pair fluxes F(U_q, U_{q+m}), m = 1..3, q = 3-m .. LB+2 along each line
    for (int t = tid; t < NP; t += NT) {
        const int line = t / PC::PL, kk = t % PC::PL;
        int m, q;
        if (kk < LB + 1) { m = 1; q = 2 + kk; }
        else if (kk < 2 * LB + 3) { m = 2; q = 1 + (kk - LB - 1); }
        else { m = 3; q = kk - 2 * LB - 3; }
        const int l = line * LS + q, r = l + m;
        const double nx = 0.5 * (S[G_NX * NB + l] + S[G_NX * NB + r]);
        const double ny = 0.5 * (S[G_NY * NB + l] + S[G_NY * NB + r]);
        const double nz = 0.5 * (S[G_NZ * NB + l] + S[G_NZ * NB + r]);
        const double xt = 0.5 * (S[G_XT * NB + l] + S[G_XT * NB + r]);
        double f[5];
        pair_flux3(S, NB, l, r, nx, ny, nz, xt, P.gas, f);
#pragma unroll
        for (int c = 0; c < 5; ++c) PB[c * NP + t] = f[c];
    }
    __syncthreads();

    // ---- D: face fluxes at q+1/2, q = 2 .. LB+2
    for (int t = tid; t < NFc; t += NT) {
        const int line = t / (LB + 1), f = t % (LB + 1);
        const int q = 2 + f;
        const int pbase = line * PC::PL;
        const int base = line * LS;
        double F[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        double FJ = 0.0;
#pragma unroll
        for (int m = 1; m <= 3; ++m) {
            const int off = m == 1 ? 0 : (m == 2 ? LB + 1 : 2 * LB + 3);
            const double al = ec_alpha(m);
            for (int s = 0; s < m; ++s) {
                const int qq = q - s;
                const int pi = pbase + off + (qq - (3 - m));
#pragma unroll
                for (int c = 0; c < 5; ++c) F[c] += al * PB[c * NP + pi];
                FJ += al * 0.5 * (S[G_XT * NB + base + qq] + S[G_XT * NB + base + qq + m]);
            }
        }
        if (P.diss) {
            const int l = base + q;
            const double nx = 0.5 * (S[G_NX * NB + l] + S[G_NX * NB + l + 1]);
            const double ny = 0.5 * (S[G_NY * NB + l] + S[G_NY * NB + l + 1]);
            const double nz = 0.5 * (S[G_NZ * NB + l] + S[G_NZ * NB + l + 1]);
            const double xtf = 0.5 * (S[G_XT * NB + l] + S[G_XT * NB + l + 1]);
            double d[5];
            face_dissipation3(S, NB, l, nx, ny, nz, xtf, P.gas, P.weno, d, P.status);
#pragma unroll
            for (int c = 0; c < 5; ++c) F[c] += d[c];
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) FB[c * NFc + t] = F[c];
        FB[5 * NFc + t] = FJ;
    }
    __syncthreads();

    // ---- E: divergence at the pencil's nodes, accumulated over the directions; the last
    // direction writes the right-hand sides or the Shu-Osher combination
    const double inv = g.inv_dxi[K];
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
        // every global operand of the node is loaded before the first global store (a store may alias a later
        // load as far as the compiler knows, which would serialise one round trip per component)
        double rh[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        double un[6], us[6];
        if (!P.first) {
#pragma unroll
            for (int c = 0; c < 6; ++c) rh[c] = P.RH[c * N + id];
        }
        const bool combine = P.last && P.mode != 1;
        if (combine) {
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                un[c] = P.JUn[c * N + id];
                us[c] = P.JUs[c * N + id];
            }
            un[5] = P.Jn[id];
            us[5] = P.Js[id];
        }
        double acc[6];
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
            for (int c = 0; c < 5; ++c) P.JUo[c * N + id] = acc[c];
            P.Jo[id] = acc[5];
        } else {
#pragma unroll
            for (int c = 0; c < 5; ++c) P.JUo[c * N + id] = P.ca * un[c] + P.cb * (us[c] + dt * acc[c]);
            const double Jnew = P.ca * un[5] + P.cb * (us[5] + dt * acc[5]);
            P.Jo[id] = Jnew;
            if (!(Jnew > 0.0)) raise_error(P.status, ES_ERR_MESH, int(id));
        }
    }
}

// pencil shapes (nodes along xi_K x lines, threads >= faces): 16 x 16 / 288 (one CTA per SM by
// shared memory), 16 x 8 / 160 (two CTAs per SM: one CTA's loads overlap the other's arithmetic),
// 16 x 4 / 96 (three CTAs per SM), 32 x 4 / 160 (two per SM, 19% halo nodes instead of 38%)
template <int K, int LB, int W, int NT>
static cudaError_t dir_prepare_shape() {
    return cudaFuncSetAttribute(k3_dir<K, LB, W, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(Pencil<LB, W>::SMEM));
}

template <int K>
static cudaError_t dir_prepare() {
    cudaError_t e = dir_prepare_shape<K, 16, 16, 288>();
    if (e == cudaSuccess) e = dir_prepare_shape<K, 16, 8, 160>();
    if (e == cudaSuccess) e = dir_prepare_shape<K, 16, 4, 96>();
    if (e == cudaSuccess) e = dir_prepare_shape<K, 32, 4, 160>();
    return e;
}

template <int K, int LB, int W, int NT>
static cudaError_t dir_launch_shape(const Dir3Params& P, cudaStream_t s) {
    const Grid3& g = P.g;
    const int nA = K == 0 ? g.n[1] : g.n[0];
    const int nB = K == 2 ? g.n[1] : g.n[2];
    const long long blocks = (long long)((g.n[K] + LB - 1) / LB) * ((nA + W - 1) / W) * nB;
    k3_dir<K, LB, W, NT><<<unsigned(blocks), NT, Pencil<LB, W>::SMEM, s>>>(P);
    return cudaGetLastError();
}

template <int K>
static cudaError_t dir_launch(const Dir3Params& P, int shape, cudaStream_t s) {
    switch (shape) {
        case 1: return dir_launch_shape<K, 16, 8, 160>(P, s);
        case 2: return dir_launch_shape<K, 16, 4, 96>(P, s);
        case 3: return dir_launch_shape<K, 32, 4, 160>(P, s);
        default: return dir_launch_shape<K, 16, 16, 288>(P, s);
    }
}

// ================================================================ CFL (eq. cfl)
// max_i sum_k (|J xi_{k,t} + n_k . v| + |n_k| c) / (J dxi_k), J xi_{k,t} = -xdot . n_k (eq. VCLCoeff), from the
// node fields and metrics of x^n; xdot = nullptr is a mesh at rest.  The maximum goes to d->red[slot].
__global__ void k3_cfl(Grid3 g, Gas G, const double* NF, const double* J, const double* NK0, const double* NK1,
                       const double* NK2, const double* xdot, int slot, DevScalars* d) {
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    const size_t M[3] = {size_t(g.n[0] + 6) * g.n[1] * g.n[2], size_t(g.n[0]) * (g.n[1] + 6) * g.n[2],
                         size_t(g.n[0]) * g.n[1] * (g.n[2] + 6)};
    const double* NK[3] = {NK0, NK1, NK2};
    double mx = 0.0;
    for (size_t id = blockIdx.x * size_t(blockDim.x) + threadIdx.x; id < N; id += size_t(gridDim.x) * blockDim.x) {
        const int i1 = int(id % g.n[0]), i2 = int((id / g.n[0]) % g.n[1]), i3 = int(id / (size_t(g.n[0]) * g.n[1]));
        const double rho = NF[G_RHO * N + id], T = NF[G_T * N + id], iom = NF[G_IOM * N + id];
        const double v[3] = {NF[G_V1 * N + id], NF[G_V2 * N + id], NF[G_V3 * N + id]};
        const double c2 = (1.0 + G.delta) * G.R * T * (iom * iom) - 2.0 * G.a * rho;
        const double c = sqrt(fmax(c2, 0.0));
        const double iJ = rcp_nr(J[id]);
        const double xd[3] = {xdot ? xdot[id] : 0.0, xdot ? xdot[N + id] : 0.0, xdot ? xdot[2 * N + id] : 0.0};
        double tot = 0.0;
        for (int k = 0; k < 3; ++k) {
            const int m1 = g.n[0] + (k == 0 ? 6 : 0), m2 = g.n[1] + (k == 1 ? 6 : 0);
            const size_t mi = (size_t(i3 + (k == 2 ? 3 : 0)) * m2 + i2 + (k == 1 ? 3 : 0)) * m1 + i1 + (k == 0 ? 3 : 0);
            const double n0 = NK[k][mi], n1 = NK[k][M[k] + mi], n2 = NK[k][2 * M[k] + mi];
            const double xt = -(xd[0] * n0 + xd[1] * n1 + xd[2] * n2);
            tot += (fabs(xt + (n0 * v[0] + n1 * v[1] + n2 * v[2])) + sqrt(n0 * n0 + n1 * n1 + n2 * n2) * c) * iJ *
                   g.inv_dxi[k];
        }
        if (!(c2 > 0.0)) tot = 1e300;
        mx = fmax(mx, tot);
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) atomic_max_pos(&d->red[slot], mx);
}

// ================================================================ init
__global__ void k3_init_J(Grid3 g, const double* x, double* J) {
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    for (size_t id = blockIdx.x * size_t(blockDim.x) + threadIdx.x; id < N; id += size_t(gridDim.x) * blockDim.x) {
        const int ii[3] = {int(id % g.n[0]), int((id / g.n[0]) % g.n[1]), int(id / (size_t(g.n[0]) * g.n[1]))};
        double Dm[3][3];                                     // Dm[c][k] = delta_k[x_c] / dxi_k
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
#pragma unroll
                for (int m = 1; m <= 3; ++m) {
                    int p[3] = {ii[0], ii[1], ii[2]}, q[3] = {ii[0], ii[1], ii[2]};
                    p[k] += m;
                    q[k] -= m;
                    s += 0.5 * ec_alpha(m) * (ghost_value3(g, x + c * N, nullptr, 0.0, p[0], p[1], p[2], c) -
                                              ghost_value3(g, x + c * N, nullptr, 0.0, q[0], q[1], q[2], c));
                }
                Dm[c][k] = s * g.inv_dxi[k];
            }
        J[id] = Dm[0][0] * (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) -
                Dm[0][1] * (Dm[1][0] * Dm[2][2] - Dm[1][2] * Dm[2][0]) +
                Dm[0][2] * (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]);
    }
}

// ================================================================ mesh (Sec. 4)
__global__ void k3_mon_terms(Grid3 g, MonitorParams mp, const double* rhoF, const double* GF, double* t0,
                             double* t1, double* t2, DevScalars* d) {
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    double m0 = 0.0, m1 = 0.0, m2 = 0.0;
    for (size_t id = blockIdx.x * size_t(blockDim.x) + threadIdx.x; id < N; id += size_t(gridDim.x) * blockDim.x) {
        const int i1 = int(id % g.n[0]), i2 = int((id / g.n[0]) % g.n[1]), i3 = int(id / (size_t(g.n[0]) * g.n[1]));
        double gr = 0.0, gg = 0.0, lg = 0.0, lr = 0.0;
        const int ii[3] = {i1, i2, i3};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double h = g.inv_dxi[k];
            const size_t ip = nb_index(g, id, ii[k], k, 1), im = nb_index(g, id, ii[k], k, -1);
            const double rp = rhoF[ip], rm = rhoF[im];
            const double Gp = GF[ip], Gm = GF[im];
            const double r0 = rhoF[id], G0 = GF[id];
            const double a = (rp - rm) * 0.5 * h, bb = (Gp - Gm) * 0.5 * h;
            const double c = (Gp - 2.0 * G0 + Gm) * h * h, e = (rp - 2.0 * r0 + rm) * h * h;
            gr += a * a;
            gg += bb * bb;
            lg += c * c;
            lr += e * e;
        }
        double v0, v1, v2;
        if (mp.kind == ES_MONITOR_SMOOTH) {
            v0 = sqrt(gr);
            v1 = 0.0;
            v2 = sqrt(lr);
        } else {
            v0 = gr;
            v1 = mp.kappa >= 2 ? gg : 0.0;
            v2 = lg;
        }
        t0[id] = v0;
        t1[id] = v1;
        t2[id] = v2;
        m0 = fmax(m0, v0);
        m1 = fmax(m1, v1);
        m2 = fmax(m2, v2);
    }
    m0 = block_max(m0);
    m1 = block_max(m1);
    m2 = block_max(m2);
    if (threadIdx.x == 0) {
        atomic_max_pos(&d->red[RED_MON0], m0);
        atomic_max_pos(&d->red[RED_MON1], m1);
        atomic_max_pos(&d->red[RED_MON2], m2);
    }
}

// omega_i <- sum_{j in {0,+-1}^3} (1/2)^(|j|_1 + 3) omega_{i+j}
__global__ void k3_filter(Grid3 g, const double* in, double* out) {
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    for (size_t id = blockIdx.x * size_t(blockDim.x) + threadIdx.x; id < N; id += size_t(gridDim.x) * blockDim.x) {
        const int i1 = int(id % g.n[0]), i2 = int((id / g.n[0]) % g.n[1]), i3 = int(id / (size_t(g.n[0]) * g.n[1]));
        // offsets of the neighbours along each direction (ghosts by copy / wrap, per direction)
        long long o1[3], o2[3], o3[3];
        o1[1] = o2[1] = o3[1] = 0;
        o1[0] = (long long)nb_index(g, id, i1, 0, -1) - (long long)id;
        o1[2] = (long long)nb_index(g, id, i1, 0, 1) - (long long)id;
        o2[0] = (long long)nb_index(g, id, i2, 1, -1) - (long long)id;
        o2[2] = (long long)nb_index(g, id, i2, 1, 1) - (long long)id;
        o3[0] = (long long)nb_index(g, id, i3, 2, -1) - (long long)id;
        o3[2] = (long long)nb_index(g, id, i3, 2, 1) - (long long)id;
        double s = 0.0;
#pragma unroll
        for (int d3 = 0; d3 < 3; ++d3) {
            double pl = 0.0;
#pragma unroll
            for (int d2 = 0; d2 < 3; ++d2) {
                double row = 0.0;
#pragma unroll
                for (int d1 = 0; d1 < 3; ++d1) row += (d1 == 1 ? 0.5 : 0.25) * in[(long long)id + o1[d1] + o2[d2] + o3[d3]];
                pl += (d2 == 1 ? 0.5 : 0.25) * row;
            }
            s += (d3 == 1 ? 0.5 : 0.25) * pl;
        }
        out[id] = s;
    }
}

// Coordinate component c of a boundary node that does not move: every component on an outflow
// end, the normal one on a wall or symmetry end (the node slides along the plane).
__device__ __forceinline__ bool fixed3(const Grid3& g, const int* ii, int c) {
    bool f = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (g.bc[k] == ES_BC_PERIODIC) continue;
        const bool lo = ii[k] == 0, hi = ii[k] == g.n[k] - 1;
        if (!lo && !hi) continue;
        const bool mir = end_mirrored(g.bc[k], lo);
        f = f || !mir || c == k;
    }
    return f;
}

// Jacobi sweep k (no warm start in 3D: sweep 0 reads x_n and writes xa, sweep k reads
// buf[(k - 1) % 2] and writes buf[k % 2]); with `check` the last block to finish compares the
// grid's max change with eps and latches convergence, after which the remaining sweeps return
__global__ void k3_jacobi(Grid3 g, const double* omega, const double* xn, double* xa, double* xb, int k,
                          DevScalars* d, int check, double eps) {
    if (d->conv) return;
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    const double* xin = k == 0 ? xn : (((k - 1) & 1) ? xb : xa);
    double* xout = (k & 1) ? xb : xa;
    double chg = 0.0;
    for (size_t id = blockIdx.x * size_t(blockDim.x) + threadIdx.x; id < N; id += size_t(gridDim.x) * blockDim.x) {
        const int ii[3] = {int(id % g.n[0]), int((id / g.n[0]) % g.n[1]), int(id / (size_t(g.n[0]) * g.n[1]))};
        const double w0 = omega[id];
        double den = 0.0, num[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
            const double ih2 = g.inv_dxi[kk] * g.inv_dxi[kk];
            const double wp = 0.5 * (w0 + omega[nb_index(g, id, ii[kk], kk, 1)]) * ih2;
            const double wm = 0.5 * (w0 + omega[nb_index(g, id, ii[kk], kk, -1)]) * ih2;
            den += wp + wm;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double xp = nb_coord(g, xin + c * N, id, ii[kk], kk, 1, c);
                const double xq = nb_coord(g, xin + c * N, id, ii[kk], kk, -1, c);
                num[c] += wp * xp + wm * xq;
            }
        }
        const double iden = rcp_nr(den);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double xv = fixed3(g, ii, c) ? xin[c * N + id] : num[c] * iden;
            chg = fmax(chg, fabs(xv - xin[c * N + id]));
            xout[c * N + id] = xv;
        }
    }
    if (check) {
        chg = block_max(chg);
        if (threadIdx.x == 0) {
            atomic_max_pos(&d->red[RED_JAC], chg);
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

// Delta_gamma over all nodes and directions (Sec. 4)
__global__ void k3_limiter(Grid3 g, const double* xn, const double* xa, const double* xb, DevScalars* d) {
    const size_t N = size_t(g.n[0]) * g.n[1] * g.n[2];
    const double* xit = d->sweeps == 0 ? xn : (((d->sweeps - 1) & 1) ? xb : xa);
    double m = 1.0;
    for (size_t id = blockIdx.x * size_t(blockDim.x) + threadIdx.x; id < N; id += size_t(gridDim.x) * blockDim.x) {
        const int ii[3] = {int(id % g.n[0]), int((id / g.n[0]) % g.n[1]), int(id / (size_t(g.n[0]) * g.n[1]))};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double dx = xit[k * N + id] - xn[k * N + id];
            if (dx < 0.0)
                m = fmin(m, div_nr(-(xn[k * N + id] - nb_coord(g, xn + k * N, id, ii[k], k, -1, k)), 2.0 * dx));
            else if (dx > 0.0)
                m = fmin(m, div_nr(nb_coord(g, xn + k * N, id, ii[k], k, 1, k) - xn[k * N + id], 2.0 * dx));
        }
    }
    m = block_min(m);
    if (threadIdx.x == 0) atomic_min_pos(&d->red[RED_GAMMA], m);
}

// ================================================================ host side
cudaError_t d3_alloc(Ctx3* d) {
    const Grid3& g = d->g;
    d->N = size_t(g.n[0]) * g.n[1] * g.n[2];
    d->NE = size_t(g.n[0] + 6) * (g.n[1] + 6) * (g.n[2] + 6);
    for (int k = 0; k < 3; ++k) d->NKk[k] = d->N / g.n[k] * (g.n[k] + 6);
    cudaError_t e = cudaMalloc((void**)&d->XE, sizeof(double) * 3 * d->NE);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->D, sizeof(double) * 9 * d->NE);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMalloc((void**)&d->NK[k], sizeof(double) * 3 * d->NKk[k]);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->NF, sizeof(double) * F3_COUNT * d->N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->RH, sizeof(double) * 6 * d->N);
    if (e == cudaSuccess && d->mixed) e = cudaMalloc((void**)&d->XD, sizeof(float) * 3 * d->NE);
    return e;
}

void d3_free(Ctx3* d) {
    if (!d) return;
    void* b[] = {d->XE, d->D, d->NK[0], d->NK[1], d->NK[2], d->NF, d->RH, d->XD};
    for (void* p : b)
        if (p) cudaFree(p);
}

cudaError_t d3_prepare() {
    cudaError_t e = dir_prepare<0>();
    if (e == cudaSuccess) e = dir_prepare<1>();
    if (e == cudaSuccess) e = dir_prepare<2>();
    return e;
}

int d3_init_J(const Ctx3* d, const double* x, void* J, cudaStream_t s, cudaError_t* err) {
    int n = 1;
    if (d->mixed) {                                   // FP64 J into the scratch, then split
        k3_init_J<<<d->grid, 256, 0, s>>>(d->g, x, d->RH);
        n += d3f_init_J(const_cast<Ctx3*>(d), d->RH, J, s);
    } else {
        k3_init_J<<<d->grid, 256, 0, s>>>(d->g, x, (double*)J);
    }
    *err = cudaGetLastError();
    return *err == cudaSuccess ? n : -1;
}

// metrics of x_s = xn + cst dt xdot for the three directions
static int enqueue_metrics(Ctx3* d, const double* xn, const double* xdot, double cst, const double* dt_dev,
                           double dt_host, cudaStream_t s, const Stage3* inc = nullptr) {
    if (d->mixed) return d3f_metrics(d, xn, xdot, cst, dt_dev, dt_host, s, inc);
    const int G = d->grid;
    k3_coords<<<G, 256, 0, s>>>(d->g, xn, cst != 0.0 ? xdot : nullptr, cst, dt_dev, dt_host, d->XE);
    k3_deriv<<<G, 256, 0, s>>>(d->g, d->XE, d->D);
    k3_metric<0><<<G, 256, 0, s>>>(d->g, d->D, d->NK[0]);
    k3_metric<1><<<G, 256, 0, s>>>(d->g, d->D, d->NK[1]);
    k3_metric<2><<<G, 256, 0, s>>>(d->g, d->D, d->NK[2]);
    return 5;
}

int d3_stage(Ctx3* d, const Stage3& a0, DevStatus* st, cudaStream_t s, cudaError_t* err) {
    int n = 0;
    Stage3 a = a0;
    if (d->mixed && a.xdot && !a.xd_ready) {       // the mixed kernels read xdot on the extended mesh as floats
        n += d3f_form_xd(d, a.xdot, s);
        a.xd_ready = 1;
    }
    if (!a.reuse) {
        n += enqueue_metrics(d, a.xn, a.xdot, a.cst, a.dt_dev, a.dt_host, s, a.xe_incr ? &a : nullptr);
        if (d->mixed) n += d3f_nodes(d, a.JUs, a.Js, st, s);
        else {
            k3_nodes<<<d->grid, 256, 0, s>>>(d->g, d->gas, (const double*)a.JUs, (const double*)a.Js, d->NF, st);
            ++n;
        }
    }
    if (d->mixed) {
        const int m = d3f_directions(d, a, st, s, err);
        return m < 0 ? -1 : n + m;
    }
    Dir3Params P;
    P.g = d->g;
    P.gas = d->gas;
    P.weno = d->weno;
    P.diss = d->diss;
    P.NF = d->NF;
    P.xdot = a.xdot;
    P.RH = d->RH;
    P.mode = a.mode;
    P.ca = a.ca;
    P.cb = a.cb;
    P.dt_host = a.dt_host;
    P.dt_dev = a.dt_dev;
    P.JUn = (const double*)a.JUn;
    P.Jn = (const double*)a.Jn;
    P.JUs = (const double*)a.JUs;
    P.Js = (const double*)a.Js;
    P.JUo = (double*)a.JUo;
    P.Jo = (double*)a.Jo;
    P.status = st;
    cudaError_t e = cudaGetLastError();
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        P.NK = d->NK[k];
        P.first = k == 0;
        P.last = k == 2;
        e = k == 0 ? dir_launch<0>(P, d->shape, s) : (k == 1 ? dir_launch<1>(P, d->shape, s) : dir_launch<2>(P, d->shape, s));
        ++n;
    }
    *err = e;
    return e == cudaSuccess ? n : -1;
}

int d3_cfl(Ctx3* d, const void* JU, const void* J, const double* x, DevScalars* dv, cudaStream_t s,
           cudaError_t* err) {
    int n = enqueue_metrics(d, x, nullptr, 0.0, nullptr, 0.0, s);
    if (d->mixed) {
        n += d3f_nodes(d, JU, J, &dv->status, s);
        n += d3f_cfl(d, J, nullptr, RED_CFL, dv, s);
    } else {
        k3_nodes<<<d->grid, 256, 0, s>>>(d->g, d->gas, (const double*)JU, (const double*)J, d->NF, &dv->status);
        k3_cfl<<<d->grid, 256, 0, s>>>(d->g, d->gas, d->NF, (const double*)J, d->NK[0], d->NK[1], d->NK[2], nullptr,
                                       RED_CFL, dv);
        n += 2;
    }
    *err = cudaGetLastError();
    return *err == cudaSuccess ? n : -1;
}

int d3_cfl_moving(Ctx3* d, const void* J, const double* xdot, DevScalars* dv, cudaStream_t s, cudaError_t* err) {
    int n;
    if (d->mixed) {
        n = d3f_cfl(d, J, xdot, RED_CFL2, dv, s);
    } else {
        k3_cfl<<<d->grid, 256, 0, s>>>(d->g, d->gas, d->NF, (const double*)J, d->NK[0], d->NK[1], d->NK[2], xdot,
                                       RED_CFL2, dv);
        n = 1;
    }
    *err = cudaGetLastError();
    return *err == cudaSuccess ? n : -1;
}

int d3_mesh(Ctx3* d, const void* JU, const void* J, const double* xn, double* xdot, DevScalars* dv,
            cudaStream_t s, cudaError_t* err, bool xe_current) {
    if (d->mixed) return d3f_mesh(d, JU, J, xn, xdot, dv, s, err, xe_current);   // FP32 pipe (es_3d_mixed.cu)
    const int G = d->grid;
    // the elementwise kernels of the 1D/2D path see the 3D mesh as N nodes in a row
    GridParams flat;
    flat.dim = 3;
    flat.n1 = int(d->N);
    flat.n2 = 1;
    flat.bc[0] = flat.bc[1] = ES_BC_PERIODIC;
    flat.inv_dxi[0] = flat.inv_dxi[1] = 1.0;
    flat.period[0] = flat.period[1] = 0.0;
    grid_floats(flat);
    int n = 0;
    launch_mon_fields(flat, d->gas, JU, J, d->rhoF, d->GF, false, G, s);
    k3_mon_terms<<<G, 256, 0, s>>>(d->g, d->mon, d->rhoF, d->GF, d->t0, d->t1, d->t2, dv);
    k_mon_omega<<<G, 256, 0, s>>>(flat, d->mon, d->t0, d->t1, d->t2, dv, d->om0);
    n += 3;
    double* om = d->om0;
    double* other = d->om1;
    for (int k = 0; k < d->filter_passes; ++k) {
        k3_filter<<<G, 256, 0, s>>>(d->g, om, other);
        ++n;
        double* t = om;
        om = other;
        other = t;
    }
    const int check = d->eps > 0.0;
    for (int k = 0; k < d->sweeps; ++k) {
        k3_jacobi<<<G, 256, 0, s>>>(d->g, om, xn, d->xa, d->xb, k, dv, check, d->eps);
        ++n;
    }
    k3_limiter<<<G, 256, 0, s>>>(d->g, xn, d->xa, d->xb, dv);
    k_velocity<<<G, 256, 0, s>>>(flat, xn, d->xa, d->xb, dv, xdot);
    n += 2;
    *err = cudaGetLastError();
    return *err == cudaSuccess ? n : -1;
}

}  // namespace es
