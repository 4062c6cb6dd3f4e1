// es_aux.cu -- initialisation, time step, and mesh-redistribution kernels.
//
// Sec. 3.2: initial J from the metrics' central differences.
// Sec. 5, eq. cfl: Delta t from the spectral radii (grid-wide max).
// Sec. 4: monitor with G (eq. van der Waalsmonitor) or the smooth-test monitor
// (eq. van der Waalssinmonitor), low-pass filter, Jacobi sweeps of the
// discretised Winslow equation, movement limiter Delta_gamma, mesh velocity.
#include <cuda_runtime.h>

#include "es_aux.h"
#include "es_bits.cuh"
#include "es_df.cuh"
#include "es_device.cuh"

namespace es {

// ------------------------------------------------------------ helpers
// A ghost coordinate (the ghost rule: periodic wrap with the period shift, odd reflection at outflow ends, mirror
// at walls).  Kept out of line: inlined at each of a kernel's neighbour reads it made the per-node kernels' code
// long and branchy, and with one node per thread their warps stalled on instruction fetch (ncu: "no
// instruction" the top stall of the sweep and CFL kernels); only boundary nodes call it.
__device__ __noinline__ double coord_ghost(int n1, int n2, int dim, int bc0, int bc1, double per0, double per1,
                                          const double* x, int gi, int gj, int comp) {
    const size_t N = size_t(n1) * n2;
    const GhostTerms ti = ghost_terms(gi, n1, bc0, comp != 0);
    GhostTerms tj;
    if (dim == 2) tj = ghost_terms(gj, n2, bc1, comp != 1);
    else { tj.idx[0] = 0; tj.w[0] = 1.0; tj.nterm = 1; tj.q = 0; }
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)              // fixed bounds: the terms stay in registers
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (a < ti.nterm && c < tj.nterm) acc += ti.w[a] * tj.w[c] * x[comp * N + size_t(tj.idx[c]) * n1 + ti.idx[a]];
    if (comp == 0) acc += ti.q * per0;
    if (comp == 1) acc += tj.q * per1;
    return acc;
}

// (the grid's scalars go by value: a reference would put the kernel's parameter block in local memory)
__device__ __forceinline__ double coord_at(const GridParams& g, const double* x, int gi, int gj, int comp) {
    const size_t N = size_t(g.n1) * g.n2;
    if (gi >= 0 && gi < g.n1 && (g.dim == 1 || (gj >= 0 && gj < g.n2)))   // interior: a plain load
        return x[comp * N + size_t(g.dim == 2 ? gj : 0) * g.n1 + gi];
    return coord_ghost(g.n1, g.n2, g.dim, g.bc[0], g.bc[1], g.period[0], g.period[1], x, gi, gj, comp);
}

// 6th-order central difference delta_k of coordinate `comp` at node (i, j), divided by dxi_k
__device__ __forceinline__ double dcoord(const GridParams& g, const double* x, int i, int j, int comp, int k) {
    double s = 0.0;
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
        const double h = 0.5 * ec_alpha(m);
        if (k == 0) s += h * (coord_at(g, x, i + m, j, comp) - coord_at(g, x, i - m, j, comp));
        else s += h * (coord_at(g, x, i, j + m, comp) - coord_at(g, x, i, j - m, comp));
    }
    return s * g.inv_dxi[k];
}

__device__ __forceinline__ double block_reduce_max(double v) {
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

__device__ __forceinline__ double block_reduce_min(double v) {
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

// state element access: double arrays, or the mixed form's (hi, lo) float planes
// (value = hi + lo, the lo plane `plane` elements after the hi plane)
__device__ __forceinline__ double ld_state(const double* a, size_t, size_t i) { return a[i]; }
__device__ __forceinline__ double ld_state(const float* a, size_t plane, size_t i) {
    return double(a[i]) + double(a[plane + i]);
}
__device__ __forceinline__ void st_state(double* a, size_t, size_t i, double v) { a[i] = v; }
__device__ __forceinline__ void st_state(float* a, size_t plane, size_t i, double v) {
    const float hi = float(v);
    a[i] = hi;
    a[plane + i] = float(v - double(hi));
}

// ------------------------------------------------------------ init
template <class TS>
__global__ void k_init_J(GridParams g, const double* x, TS* J) {
    const int N = g.n1 * g.n2;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        if (g.dim == 1) {
            st_state(J, N, id, dcoord(g, x, i, 0, 0, 0));
        } else {
            const double x1 = dcoord(g, x, i, j, 0, 0), x2 = dcoord(g, x, i, j, 0, 1);
            const double y1 = dcoord(g, x, i, j, 1, 0), y2 = dcoord(g, x, i, j, 1, 1);
            st_state(J, N, id, x1 * y2 - x2 * y1);
        }
    }
}

template <class TS>
__global__ void k_prim_to_cons(GridParams g, Gas G, const double* rho, const double* v, const double* p,
                               const TS* J, TS* JU) {
    const int N = g.n1 * g.n2;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const double r = rho[id];
        const double T = (p[id] + G.a * r * r) * (1.0 - G.b * r) / (G.R * r);
        double ke = 0.0;
        for (int k = 0; k < g.dim; ++k) ke += v[k * N + id] * v[k * N + id];
        const double E = r * (G.cv * T - G.a * r) + 0.5 * r * ke;
        const double Jv = ld_state(J, N, id);
        const size_t P = size_t(g.dim + 2) * N;
        st_state(JU, P, id, Jv * r);
        for (int k = 0; k < g.dim; ++k) st_state(JU, P, (1 + k) * N + id, Jv * r * v[k * N + id]);
        st_state(JU, P, (1 + g.dim) * N + id, Jv * E);
    }
}

// ------------------------------------------------------------ time step
__global__ void k_reset(DevScalars* d) {
    if (threadIdx.x == 0 && blockIdx.x == 0) reset_scalars(d);
}

// eq. cfl: max_i sum_k (|J xi_{k,t} + n_k . v| + |n_k| c) / (J dxi_k) with J xi_{k,t} = -xdot . n_k
// (eq. VCLCoeff); xdot = nullptr is a mesh at rest.  The maximum goes to d->red[slot].
template <class TS>
__global__ void k_cfl(GridParams g, Gas G, const TS* JU, const TS* J, const double* x, const double* xdot, int slot,
                      DevScalars* d, double* t0, double* t1, double* rhoF, double* GF, int set_dt, double cfl,
                      double dt_fixed) {
    const int N = g.n1 * g.n2;
    double m = 0.0;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        const size_t P = size_t(g.dim + 2) * N;
        const double iJ = rcp_nr(ld_state(J, N, id));
        const double rho = ld_state(JU, P, id) * iJ;
        const double irho = rcp_nr(rho);
        const double v1 = ld_state(JU, P, N + id) * iJ * irho;
        const double v2 = g.dim == 2 ? ld_state(JU, P, 2 * N + id) * iJ * irho : 0.0;
        const double E = ld_state(JU, P, (g.dim + 1) * N + id) * iJ;
        const double T = (E * irho - 0.5 * (v1 * v1 + v2 * v2) + G.a * rho) * G.icv;
        const double om = 1.0 - G.b * rho;
        const double iom = rcp_nr(om);
        const double c2 = (1.0 + G.delta) * G.R * T * (iom * iom) - 2.0 * G.a * rho;
        if (rhoF) {                     // the monitor's fields from the same node state (k_mon_fields' formulas)
            const double pnn3 = (1.0 + G.delta) * (2.0 + G.delta) * G.R * T * (iom * iom * iom) - 6.0 * G.a * rho;
            rhoF[id] = rho;
            GF[id] = div_nr(pnn3, 2.0 * c2);
        }
        const double c = sqrt(fmax(c2, 0.0));
        const double xd1 = xdot != nullptr ? xdot[id] : 0.0;
        double tot;
        const bool ok = c2 > 0.0;
        if (g.dim == 1) {
            tot = (fabs(-xd1 + v1) + c) * iJ * g.inv_dxi[0];
            if (t0) {
                const double f = iJ * g.inv_dxi[0];
                t0[id] = v1 * f;
                t0[N + id] = f;
                t0[2 * N + id] = ok ? c * f : 1e300;
            }
        } else {
            const double xd2 = xdot != nullptr ? xdot[N + id] : 0.0;
            const double x1 = dcoord(g, x, i, j, 0, 0), x2 = dcoord(g, x, i, j, 0, 1);
            const double y1 = dcoord(g, x, i, j, 1, 0), y2 = dcoord(g, x, i, j, 1, 1);
            const double a1 = y2, b1 = -x2;          // J dxi_1/dx
            const double a2 = -y1, b2 = x1;          // J dxi_2/dx
            const double tx1 = -(xd1 * a1 + xd2 * b1), tx2 = -(xd1 * a2 + xd2 * b2);     // J xi_{k,t}
            const double n1c = sqrt(a1 * a1 + b1 * b1) * c, n2c = sqrt(a2 * a2 + b2 * b2) * c;
            tot = (fabs(tx1 + (a1 * v1 + b1 * v2)) + n1c) * iJ * g.inv_dxi[0] +
                  (fabs(tx2 + (a2 * v1 + b2 * v2)) + n2c) * iJ * g.inv_dxi[1];
            if (t0) {
                const double f1 = iJ * g.inv_dxi[0], f2 = iJ * g.inv_dxi[1];
                t0[id] = (a1 * v1 + b1 * v2) * f1;
                t0[N + id] = a1 * f1;
                t0[2 * N + id] = b1 * f1;
                t0[3 * N + id] = ok ? n1c * f1 : 1e300;
                t1[id] = (a2 * v1 + b2 * v2) * f2;
                t1[N + id] = a2 * f2;
                t1[2 * N + id] = b2 * f2;
                t1[3 * N + id] = ok ? n2c * f2 : 0.0;
            }
        }
        if (!ok) tot = 1e300;
        m = fmax(m, tot);
    }
    m = block_reduce_max(m);
    if (threadIdx.x == 0) {
        atomic_max_pos(&d->red[slot], m);
        if (set_dt) {                   // k_dt's work, by the last block to finish
            __threadfence();
            const unsigned int ticket = atomicAdd(&d->done, 1u);
            if (ticket == gridDim.x - 1) {
                set_dt_from_max(d, __longlong_as_double((long long)atomicAdd(&d->red[slot], 0ULL)), cfl, dt_fixed);
                d->done = 0u;
            }
        }
    }
}

// Delta t = CFL / max (or the fixed step), clipped to t_end; 0 once t_end is reached
__global__ void k_dt(DevScalars* d, double cfl, double dt_fixed) {
    if (threadIdx.x == 0 && blockIdx.x == 0) set_dt_from_cfl(d, cfl, dt_fixed);
}

// Delta t_n = min(Delta t^(0), CFL / the maximum with the step's mesh velocity)
__global__ void k_dt_moving(DevScalars* d, double cfl) {
    if (threadIdx.x == 0 && blockIdx.x == 0) shrink_dt_for_mesh(d, cfl);
}

__global__ void k_set_dt(DevScalars* d, double dt) {
    if (threadIdx.x == 0 && blockIdx.x == 0) d->dt = dt;
}

__global__ void k_set_t_end(DevScalars* d, double t_end) {
    if (threadIdx.x == 0 && blockIdx.x == 0) d->t_end = t_end;
}

// the float displacement x - (x_00 + i dxi_1) of one coordinate, in double-float arithmetic on the FP32 pipe:
// x and x_00 split from their bits (es_bits.cuh), i dxi_1 an exact product plus i dxl, error-free sums; the
// absolute error is about 2^-45 |x|, far below the float rounding of the displacement itself
__device__ __forceinline__ float disp_f32(double x, float x0h, float x0l, int i, float dh, float dl) {
    float xh, xl;
    bits::split(x, xh, xl);
    const float fi = bits::small_int(i);
    const float ph = fi * dh;
    const float pl = fmaf(fi, dl, fmaf(fi, dh, -ph));
    // b = x_00 + i dxi as (bh, bl)
    const float bh = x0h + ph;
    const float bv = bh - x0h;
    const float bl = ((x0h - (bh - bv)) + (ph - bv)) + (x0l + pl);
    // x - b
    const float sh = xh - bh;
    const float sv = sh - xh;
    const float se = (xh - (sh - sv)) + (-bh - sv);
    return sh + (se + (xl - bl));
}

__global__ void k_advance(GridParams g, double* x, const double* xdot, DevScalars* d, float* fdisp, int reset) {
    const int N = g.n1 * g.n2;
    const double dt = d->dt;
    const bool move = xdot != nullptr && dt != 0.0;
    if (fdisp) {
        float b0h, b0l, b1h = 0.0f, b1l = 0.0f;
        bits::split(d->base[0], b0h, b0l);
        if (g.dim == 2) bits::split(d->base[1], b1h, b1l);
        for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < g.dim * N; id += gridDim.x * blockDim.x) {
            const double v = move ? x[id] + dt * xdot[id] : x[id];
            if (move) x[id] = v;
            const int c = id < N ? 0 : 1, node = id - c * N;
            const int i = node % g.n1, j = node / g.n1;
            fdisp[id] = c == 0 ? disp_f32(v, b0h, b0l, i, g.dxh[0], g.dxl[0]) : disp_f32(v, b1h, b1l, j, g.dxh[1], g.dxl[1]);
        }
    } else if (move) {
        for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < g.dim * N; id += gridDim.x * blockDim.x)
            x[id] += dt * xdot[id];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d->t += dt;
        d->last_dt = dt;
        if (reset) reset_scalars(d);
    }
}

// ------------------------------------------------------------ entropy production (FP64)
// Knuth's error-free sum: s + e == a + b exactly
__device__ __forceinline__ void two_sum_d(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (s, e) += (s2, e2) for compensated sums
__device__ __forceinline__ void add_comp(double& s, double& e, double s2, double e2) {
    double t, err;
    two_sum_d(s, s2, t, err);
    s = t;
    e += e2 + err;
}

// Per node the rate of J eta (eta = -rho s): V . d(JU)/dt - phi dJ/dt, with the entropy variables
// V = ((e + p/rho)/T - s - |v|^2/(2T), v/T, -1/T) (Sec. 2, general units) and phi = p/T.  Each block
// writes the compensated sum of its nodes' terms and the sum of their magnitudes to part[3 b ..]; the
// grid-stride order and the tree below are fixed, so the result does not change from run to run.
template <class TS>
__global__ void k_entropy_terms(int N, int dim, Gas G, const TS* JU, const TS* J, const TS* dJU, const TS* dJ,
                                double* part) {
    __shared__ double sh[3][256];
    const size_t P = size_t(dim + 2) * N;
    double s = 0.0, e = 0.0, a = 0.0;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const double Jv = ld_state(J, N, id);
        const double rho = ld_state(JU, P, id) / Jv;
        double v[3] = {0.0, 0.0, 0.0}, v2 = 0.0;
        for (int k = 0; k < dim; ++k) {
            v[k] = ld_state(JU, P, size_t(1 + k) * N + id) / Jv / rho;
            v2 += v[k] * v[k];
        }
        const double E = ld_state(JU, P, size_t(dim + 1) * N + id) / Jv;
        const double T = (E / rho - 0.5 * v2 + G.a * rho) / G.cv;
        const double om = 1.0 - G.b * rho;
        const double sent = G.cv * log(T) + G.R * log(om / rho);
        const double V0 = G.cv - sent - 2.0 * G.a * rho / T + G.R / om - 0.5 * v2 / T;
        const double p = rho * G.R * T / om - G.a * rho * rho;
        double term = V0 * ld_state(dJU, P, id);
        for (int k = 0; k < dim; ++k) term += v[k] / T * ld_state(dJU, P, size_t(1 + k) * N + id);
        term += -1.0 / T * ld_state(dJU, P, size_t(dim + 1) * N + id);
        term -= p / T * ld_state(dJ, N, id);
        add_comp(s, e, term, 0.0);
        a += fabs(term);
    }
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = e;
    sh[2][threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            double s1 = sh[0][threadIdx.x], e1 = sh[1][threadIdx.x];
            add_comp(s1, e1, sh[0][threadIdx.x + w], sh[1][threadIdx.x + w]);
            sh[0][threadIdx.x] = s1;
            sh[1][threadIdx.x] = e1;
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = sh[0][0];
        part[3 * blockIdx.x + 1] = sh[1][0];
        part[3 * blockIdx.x + 2] = sh[2][0];
    }
}

// the blocks' partial sums in block order; out = (vol sum, vol sum of magnitudes)
__global__ void k_entropy_sum(int nb, const double* part, double vol, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0, e = 0.0, a = 0.0;
    for (int b = 0; b < nb; ++b) {
        add_comp(s, e, part[3 * b], part[3 * b + 1]);
        a += part[3 * b + 2];
    }
    out[0] = vol * (s + e);
    out[1] = vol * a;
}

// ------------------------------------------------------------ monitor (Sec. 4)
// density and fundamental derivative G = nu^3 p_nunu|_s / (2 c^2) at the nodes
template <class TS>
__global__ void k_mon_fields(GridParams g, Gas G, const TS* JU, const TS* J, double* rhoF, double* GF) {
    const int N = g.n1 * g.n2;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const size_t P = size_t(g.dim + 2) * N;
        const double iJ = rcp_nr(ld_state(J, N, id));
        const double rho = ld_state(JU, P, id) * iJ;
        const double irho = rcp_nr(rho);
        double ke = 0.0;
        for (int k = 0; k < g.dim; ++k) {
            const double v = ld_state(JU, P, (1 + k) * N + id) * iJ * irho;
            ke += v * v;
        }
        const double E = ld_state(JU, P, (g.dim + 1) * N + id) * iJ;
        const double T = (E * irho - 0.5 * ke + G.a * rho) * G.icv;
        const double om = 1.0 - G.b * rho;
        const double iom = rcp_nr(om);
        const double c2 = (1.0 + G.delta) * G.R * T * (iom * iom) - 2.0 * G.a * rho;
        const double pnn3 = (1.0 + G.delta) * (2.0 + G.delta) * G.R * T * (iom * iom * iom) - 6.0 * G.a * rho;
        rhoF[id] = rho;
        GF[id] = div_nr(pnn3, 2.0 * c2);
    }
}

__device__ __forceinline__ double field_at(const GridParams& g, const double* f, int i, int j) {
    const int si = state_index(i, g.n1, g.bc[0]);
    const int sj = g.dim == 2 ? state_index(j, g.n2, g.bc[1]) : 0;
    return f[sj * g.n1 + si];
}

// raw monitor terms and their grid maxima
__global__ void k_mon_terms(GridParams g, MonitorParams mp, const double* rhoF, const double* GF, double* t0,
                            double* t1, double* t2, DevScalars* d) {
    const int N = g.n1 * g.n2;
    double m0 = 0.0, m1 = 0.0, m2 = 0.0;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        double gr = 0.0, gg = 0.0, lg = 0.0, lr = 0.0;
        #pragma unroll
        for (int k = 0; k < 2; ++k) {          // fixed bound: the spacings are indexed by constants
            if (k >= g.dim) break;
            const int di = k == 0, dj = k == 1;
            const double h2 = g.inv_dxi[k];
            const double rp = field_at(g, rhoF, i + di, j + dj), rm = field_at(g, rhoF, i - di, j - dj);
            const double r0 = rhoF[id];
            const double Gp = field_at(g, GF, i + di, j + dj), Gm = field_at(g, GF, i - di, j - dj);
            const double G0 = GF[id];
            const double a = (rp - rm) * 0.5 * h2, b = (Gp - Gm) * 0.5 * h2;
            const double c = (Gp - 2.0 * G0 + Gm) * h2 * h2, e = (rp - 2.0 * r0 + rm) * h2 * h2;
            gr += a * a;
            gg += b * b;
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
    m0 = block_reduce_max(m0);
    m1 = block_reduce_max(m1);
    m2 = block_reduce_max(m2);
    if (threadIdx.x == 0) {
        atomic_max_pos(&d->red[RED_MON0], m0);
        atomic_max_pos(&d->red[RED_MON1], m1);
        atomic_max_pos(&d->red[RED_MON2], m2);
    }
}

__global__ void k_mon_omega(GridParams g, MonitorParams mp, const double* t0, const double* t1, const double* t2,
                            const DevScalars* d, double* omega) {
    const int N = g.n1 * g.n2;
    const double M0 = __longlong_as_double((long long)d->red[RED_MON0]);
    const double M1 = __longlong_as_double((long long)d->red[RED_MON1]);
    const double M2 = __longlong_as_double((long long)d->red[RED_MON2]);
    const double c0 = M0 > 0.0 ? mp.w0 / M0 : 0.0;
    const double c1 = M1 > 0.0 ? mp.w1 / M1 : 0.0;
    const double c2 = M2 > 0.0 ? mp.w2 / M2 : 0.0;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x)
        omega[id] = sqrt(1.0 + c0 * t0[id] + c1 * t1[id] + c2 * t2[id]);
}

// low-pass filter: omega_i <- sum_{j in {0,+-1}^d} (1/2)^(|j|_1 + d) omega_{i+j}
__global__ void k_filter(GridParams g, const double* in, double* out) {
    const int N = g.n1 * g.n2;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        double s;
        if (g.dim == 1) {
            s = 0.25 * field_at(g, in, i - 1, 0) + 0.5 * in[id] + 0.25 * field_at(g, in, i + 1, 0);
        } else {
            s = 0.0;
            for (int dj = -1; dj <= 1; ++dj) {
                double row = 0.0;
                for (int di = -1; di <= 1; ++di) {
                    const double wgt = (di == 0 ? 0.5 : 0.25);
                    row += wgt * field_at(g, in, i + di, j + dj);
                }
                s += (dj == 0 ? 0.5 : 0.25) * row;
            }
        }
        out[id] = s;
    }
}

// Result buffer of the Jacobi iteration so far: x_n before the first sweep, else
// the buffer the last sweep wrote (sweep k writes buf[(pick + k) % 2]).
__device__ __forceinline__ const double* jacobi_result(const DevScalars* d, const double* xn, const double* xa,
                                                      const double* xb) {
    if (d->sweeps == 0) return xn;
    return ((d->pick + d->sweeps - 1) & 1) ? xb : xa;
}

// Coordinate component c of a boundary node that does not move: every component on an outflow end,
// the normal one on a wall or symmetry end (the node slides along it).
__device__ __forceinline__ bool fixed_comp(const GridParams& g, int i, int j, int c) {
    bool f = false;
    if (g.bc[0] != ES_BC_PERIODIC && (i == 0 || i == g.n1 - 1)) f = !end_mirrored(g.bc[0], i == 0) || c == 0;
    if (g.dim == 2 && g.bc[1] != ES_BC_PERIODIC && (j == 0 || j == g.n2 - 1))
        f = f || !end_mirrored(g.bc[1], j == 0) || c == 1;
    return f;
}

// One Jacobi sweep of sum_k [w_{k,+} (x_{i+e_k} - x_i) - w_{k,-} (x_i - x_{i-e_k})]/dxi_k^2 = 0
// from xin into xout; returns this thread's max change
// One sweep from xin into xout; CHG: returns the largest change; LIMIT: also min-accumulates into *lim the
// limiter's bound Delta_gamma at every node from the result and x^n = xn (k_limiter's rule and arithmetic, so
// the last sweep can take the limiter's work)
template <bool CHG, bool LIMIT>
__device__ __forceinline__ double jacobi_sweep(const GridParams& g, const double* omega, const double* xin,
                                              double* xout, const double* xn = nullptr, double* lim = nullptr) {
    const int N = g.n1 * g.n2;
    double chg = 0.0, m = 1.0;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        const double w0 = omega[id];
        double den = 0.0, num[2] = {0.0, 0.0};
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {     // fixed bounds: num[] stays in registers
            if (kk >= g.dim) break;
            const int di = kk == 0, dj = kk == 1;
            const double ih2 = g.inv_dxi[kk] * g.inv_dxi[kk];
            const double wp = 0.5 * (w0 + field_at(g, omega, i + di, j + dj)) * ih2;
            const double wm = 0.5 * (w0 + field_at(g, omega, i - di, j - dj)) * ih2;
            den += wp + wm;
#pragma unroll
            for (int c = 0; c < 2; ++c)
                if (c < g.dim)
                    num[c] += wp * coord_at(g, xin, i + di, j + dj, c) + wm * coord_at(g, xin, i - di, j - dj, c);
        }
        const double iden = rcp_nr(den);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (c >= g.dim) break;
            const double xv = fixed_comp(g, i, j, c) ? xin[c * N + id] : num[c] * iden;
            if (CHG) chg = fmax(chg, fabs(xv - xin[c * N + id]));
            xout[c * N + id] = xv;
            if (LIMIT) {
                const double x0 = xn[c * N + id];
                const double dx = xv - x0;
                const int di = c == 0, dj = c == 1;
                if (dx < 0.0) m = fmin(m, div_nr(-(x0 - coord_at(g, xn, i - di, j - dj, c)), 2.0 * dx));
                else if (dx > 0.0) m = fmin(m, div_nr(coord_at(g, xn, i + di, j + dj, c) - x0, 2.0 * dx));
            }
        }
    }
    if (LIMIT) *lim = m;
    return chg;
}

// Sweep k of the iteration.  Sweep k >= 1 reads buf[(pick + k - 1) % 2] and writes
// buf[(pick + k) % 2]; sweep 0 reads `first` (x_n or the warm start) and writes buf[dst0].  Once
// the iteration has converged (d->conv) the remaining sweeps return at once.  With `check`, the
// grid-wide max change goes to red[slot]; if `decide`, the last block to finish compares it with eps.
__global__ void k_jacobi(GridParams g, const double* omega, const double* first, double* xa, double* xb, int k,
                         int dst0, DevScalars* d, int check, int slot, int decide, double eps, int limit) {
    if (d->conv) return;
    const double* xin;
    double* xout;
    if (k == 0) {
        xin = first;
        xout = dst0 ? xb : xa;
    } else {
        const int src = (d->pick + k - 1) & 1;
        xin = src ? xb : xa;
        xout = src ? xa : xb;
    }
    double chg = 0.0;
    if (check) {
        chg = jacobi_sweep<true, false>(g, omega, xin, xout);
    } else if (limit) {             // the last sweep without a tolerance: k_limiter's work (first is x^n)
        double lim = 1.0;
        jacobi_sweep<false, true>(g, omega, xin, xout, first, &lim);
        lim = block_reduce_min(lim);
        if (threadIdx.x == 0) atomic_min_pos(&d->red[RED_GAMMA], lim);
    } else {
        jacobi_sweep<false, false>(g, omega, xin, xout);
    }
    if (check) {
        chg = block_reduce_max(chg);
        if (threadIdx.x == 0) {
            atomic_max_pos(&d->red[slot], chg);
            __threadfence();
            const unsigned int ticket = atomicAdd(&d->done, 1u);
            if (ticket == gridDim.x - 1) {                 // every block's maximum is in
                if (decide) {
                    const double c = __longlong_as_double((long long)atomicAdd(&d->red[slot], 0ULL));
                    if (c < eps) d->conv = 1;
                    d->red[slot] = 0ULL;
                }
                d->done = 0u;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (k > 0 || slot == RED_JAC)) atomicAdd(&d->sweeps, 1);
}

// The body of a graph while-loop over the sweeps with a tolerance: sweep k = d->sweeps (the
// same buffers as k_jacobi), and the last block to finish tests the change, counts the sweep
// and sets the loop's condition: another sweep while not converged and fewer than mu sweeps.
__global__ void k_jacobi_loop(GridParams g, const double* omega, const double* xn, double* xa, double* xb,
                              DevScalars* d, double eps, int mu, cudaGraphConditionalHandle h) {
    if (d->conv || d->sweeps >= mu) {
        if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
        return;
    }
    const int k = d->sweeps;
    const double* xin;
    double* xout;
    if (k == 0) {
        xin = xn;
        xout = xa;
    } else {
        const int src = (d->pick + k - 1) & 1;
        xin = src ? xb : xa;
        xout = src ? xa : xb;
    }
    double chg = block_reduce_max(jacobi_sweep<true, false>(g, omega, xin, xout));
    if (threadIdx.x == 0) {
        atomic_max_pos(&d->red[RED_JAC], chg);
        __threadfence();
        const unsigned int ticket = atomicAdd(&d->done, 1u);
        if (ticket == gridDim.x - 1) {
            const double c = __longlong_as_double((long long)atomicAdd(&d->red[RED_JAC], 0ULL));
            if (c < eps) d->conv = 1;
            d->red[RED_JAC] = 0ULL;
            d->done = 0u;
            d->sweeps = k + 1;
            cudaGraphSetConditional(h, (d->conv == 0 && k + 1 < mu) ? 1u : 0u);
        }
    }
}

// Guarded warm start: the first sweep ran from x_n (into buf[0], change c0 in red[RED_JAC]) and
// from the warm start (into buf[1], change c1 in red[RED_JAC2]); keep the warm start if
// c1 < ratio c0 (ties and non-finite changes keep x_n).
__global__ void k_pick(DevScalars* d, int check, double eps, double ratio) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double c0 = __longlong_as_double((long long)d->red[RED_JAC]);
        const double c1 = __longlong_as_double((long long)d->red[RED_JAC2]);
        const int pick = (c1 < ratio * c0) ? 1 : 0;
        d->pick = pick;
        d->sweeps = 1;
        if (check && (pick ? c1 : c0) < eps) d->conv = 1;
        d->red[RED_JAC] = 0ULL;
        d->red[RED_JAC2] = 0ULL;
        d->last_change[0] = c0;
        d->last_change[1] = c1;
    }
}

// Delta_gamma: each node moves at most half of the spacing towards its neighbour (Sec. 4)
__global__ void k_limiter(GridParams g, const double* xn, const double* xa, const double* xb, DevScalars* d) {
    const int N = g.n1 * g.n2;
    const double* xit = jacobi_result(d, xn, xa, xb);
    double m = 1.0;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        for (int k = 0; k < g.dim; ++k) {
            const double dx = xit[k * N + id] - xn[k * N + id];
            const int di = k == 0, dj = k == 1;
            if (dx < 0.0) m = fmin(m, div_nr(-(xn[k * N + id] - coord_at(g, xn, i - di, j - dj, k)), 2.0 * dx));
            else if (dx > 0.0) m = fmin(m, div_nr(coord_at(g, xn, i + di, j + dj, k) - xn[k * N + id], 2.0 * dx));
        }
    }
    m = block_reduce_min(m);
    if (threadIdx.x == 0) atomic_min_pos(&d->red[RED_GAMMA], m);
}

__global__ void k_velocity(GridParams g, const double* xn, const double* xa, const double* xb, DevScalars* d,
                           double* xdot, const double* t0, const double* t1, double cfl) {
    const int N = g.n1 * g.n2;
    const double* xit = jacobi_result(d, xn, xa, xb);
    const double gam = __longlong_as_double((long long)d->red[RED_GAMMA]);
    const double dt = d->dt;
    const double f = dt > 0.0 ? gam / dt : 0.0;
    if (cfl > 0.0) {
        // per node: the velocity, then eq. cfl's term with it; the last block to finish shrinks dt
        double m = 0.0;
        for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
            const double v1 = f * (xit[id] - xn[id]);
            xdot[id] = v1;
            double v2 = 0.0;
            if (g.dim == 2) {
                v2 = f * (xit[N + id] - xn[N + id]);
                xdot[N + id] = v2;
            }
            m = fmax(m, cfl_moving_term(t0, t1, size_t(N), size_t(id), g.dim, v1, v2));
        }
        m = block_reduce_max(m);
        if (threadIdx.x == 0) {
            atomic_max_pos(&d->red[RED_CFL2], m);
            __threadfence();
            const unsigned int ticket = atomicAdd(&d->done, 1u);
            if (ticket == gridDim.x - 1) {          // every block's maximum is in: every block has read dt
                shrink_dt_to(d, __longlong_as_double((long long)atomicAdd(&d->red[RED_CFL2], 0ULL)), cfl);
                d->done = 0u;
            }
        }
    } else {
        for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < g.dim * N; id += gridDim.x * blockDim.x)
            xdot[id] = f * (xit[id] - xn[id]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d->gamma = gam;
        d->sweeps_total += d->sweeps;
        d->solves += 1;
        d->warm_kept += d->pick;
    }
}

// x_out = the Jacobi iterate (no limiter); disp = (x_out - x_n)/dxi_k as float (both nullable)
__global__ void k_jacobi_out(GridParams g, const double* xn, const double* xa, const double* xb,
                             const DevScalars* d, double* xout, float* disp) {
    const int N = g.n1 * g.n2;
    const double* xit = jacobi_result(d, xn, xa, xb);
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < g.dim * N; id += gridDim.x * blockDim.x) {
        const double v = xit[id];
        if (xout) xout[id] = v;
        if (disp) disp[id] = float((v - xn[id]) * (id < N ? g.inv_dxi[0] : g.inv_dxi[1]));
    }
}

// Features of the learned warm start (2D): ln(omega), G/(1 + |G|) and the mesh
// displacement from the Cartesian base in cells, as float planes [4][n2][n1].
__global__ void k_features(GridParams g, const double* omega, const double* GF, const double* x, float* feat) {
    const int N = g.n1 * g.n2;
    const double x00 = x[0], y00 = x[N];
    const double dxi1 = 1.0 / g.inv_dxi[0], dxi2 = 1.0 / g.inv_dxi[1];
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        const double G = GF[id];
        feat[id] = float(log(omega[id]));
        feat[N + id] = float(G / (1.0 + fabs(G)));
        feat[2 * N + id] = float((x[id] - (x00 + i * dxi1)) * g.inv_dxi[0]);
        feat[3 * N + id] = float((x[N + id] - (y00 + j * dxi2)) * g.inv_dxi[1]);
    }
}

// warm start x0 = x_n + dxi * NN (per direction); fixed nodes and non-finite outputs keep x_n
__global__ void k_warm_start(GridParams g, const double* xn, const float* out, double* x0) {
    const int N = g.n1 * g.n2;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        for (int c = 0; c < 2; ++c) {
            const float o = out[c * N + id];
            const bool ok = !fixed_comp(g, i, j, c) && isfinite(o);
            x0[c * N + id] = xn[c * N + id] + (ok ? double(o) / g.inv_dxi[c] : 0.0);
        }
    }
}

// Mixed form: FP32 displacement from the Cartesian base (x_00 + i dxi_1, y_00 + j dxi_2)
// and FP32 mesh velocity, once per step (the base is linear in the node index,
// so delta_k of it is exactly dxi_k e_k)
__global__ void k_mesh_f32(GridParams g, const double* __restrict__ x, const double* __restrict__ xdot,
                           float* __restrict__ disp, float* __restrict__ fxd, DevScalars* rst) {
    const int N = g.n1 * g.n2;
    if (rst && blockIdx.x == 0 && threadIdx.x == 0) {
        reset_scalars(rst);
        rst->base[0] = x[0];                     // the origin the step's displacement is measured from
        rst->base[1] = g.dim == 2 ? x[N] : 0.0;
    }
    float x0h, x0l, y0h = 0.0f, y0l = 0.0f;
    bits::split(x[0], x0h, x0l);
    if (g.dim == 2) bits::split(x[N], y0h, y0l);
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        disp[id] = disp_f32(x[id], x0h, x0l, i, g.dxh[0], g.dxl[0]);
        if (g.dim == 2) disp[N + id] = disp_f32(x[N + id], y0h, y0l, j, g.dxh[1], g.dxl[1]);
        if (xdot)                           // fxd is read only where a velocity was given
            for (int k = 0; k < g.dim; ++k) fxd[k * N + id] = float(xdot[k * N + id]);
    }
}

// launchers of the kernels templated on the state type (float in the mixed form)
void launch_init_J(const GridParams& g, const double* x, void* J, bool f32, int grid, cudaStream_t s) {
    if (f32) k_init_J<float><<<grid, 256, 0, s>>>(g, x, (float*)J);
    else k_init_J<double><<<grid, 256, 0, s>>>(g, x, (double*)J);
}

void launch_prim_to_cons(const GridParams& g, const Gas& G, const double* rho, const double* v, const double* p,
                         const void* J, void* JU, bool f32, int grid, cudaStream_t s) {
    if (f32) k_prim_to_cons<float><<<grid, 256, 0, s>>>(g, G, rho, v, p, (const float*)J, (float*)JU);
    else k_prim_to_cons<double><<<grid, 256, 0, s>>>(g, G, rho, v, p, (const double*)J, (double*)JU);
}

void launch_entropy_rate(int N, int dim, const Gas& G, const void* JU, const void* J, const void* dJU,
                         const void* dJ, double vol, double* part, double* out, bool f32, int grid, cudaStream_t s) {
    if (f32)
        k_entropy_terms<float><<<grid, 256, 0, s>>>(N, dim, G, (const float*)JU, (const float*)J, (const float*)dJU,
                                                    (const float*)dJ, part);
    else
        k_entropy_terms<double><<<grid, 256, 0, s>>>(N, dim, G, (const double*)JU, (const double*)J,
                                                     (const double*)dJU, (const double*)dJ, part);
    k_entropy_sum<<<1, 32, 0, s>>>(grid, part, vol, out);
}

void launch_cfl(const GridParams& g, const Gas& G, const void* JU, const void* J, const double* x,
                const double* xdot, int slot, DevScalars* d, bool f32, int grid, cudaStream_t s, double* t0,
                double* t1, int block, double* rhoF, double* GF, int set_dt, double cfl, double dt_fixed) {
    if (f32)
        k_cfl<float><<<grid, block, 0, s>>>(g, G, (const float*)JU, (const float*)J, x, xdot, slot, d, t0, t1, rhoF, GF,
                                            set_dt, cfl, dt_fixed);
    else
        k_cfl<double><<<grid, block, 0, s>>>(g, G, (const double*)JU, (const double*)J, x, xdot, slot, d, t0, t1, rhoF,
                                             GF, set_dt, cfl, dt_fixed);
}

void launch_mon_fields(const GridParams& g, const Gas& G, const void* JU, const void* J, double* rhoF, double* GF,
                       bool f32, int grid, cudaStream_t s, int block) {
    if (f32) k_mon_fields<float><<<grid, block, 0, s>>>(g, G, (const float*)JU, (const float*)J, rhoF, GF);
    else k_mon_fields<double><<<grid, block, 0, s>>>(g, G, (const double*)JU, (const double*)J, rhoF, GF);
}

}  // namespace es

namespace es {
__global__ void k_selftest_division(const double* a, const double* b, double* q, double* r, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        q[i] = div_nr(a[i], b[i]);
        r[i] = rcp_nr(b[i]);
    }
}
}  // namespace es

namespace es {
__global__ void k_selftest_mixed_arith(const double* x, const float* f, const float* a, const float* b, int64_t n,
                                       float* split, double* wide, float* mul, float* add) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        bits::split(x[i], split[2 * i], split[2 * i + 1]);
        wide[i] = bits::widen(f[i]);
        const mixed::df u = {a[2 * i], a[2 * i + 1]}, v = {b[2 * i], b[2 * i + 1]};
        const mixed::df p = mixed::df_mul(u, v), q = mixed::df_add(u, v);
        mul[2 * i] = p.hi;
        mul[2 * i + 1] = p.lo;
        add[2 * i] = q.hi;
        add[2 * i + 1] = q.lo;
    }
}
}  // namespace es

extern "C" int es_selftest_mixed_arith(const double* x, const float* f, const float* a, const float* b, int64_t n,
                                       float* split, double* wide, float* mul, float* add, void* stream) {
    if (!x || !f || !a || !b || !split || !wide || !mul || !add || n <= 0) return ES_ERR_ARG;
    const int64_t blocks = (n + 255) / 256;
    es::k_selftest_mixed_arith<<<int(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(
        x, f, a, b, n, split, wide, mul, add);
    return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}

extern "C" int es_selftest_division(const double* a, const double* b, double* q, double* r, int64_t n, void* stream) {
    if (!a || !b || !q || !r || n <= 0) return ES_ERR_ARG;
    const int64_t blocks = (n + 255) / 256;
    es::k_selftest_division<<<int(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(a, b, q, r, n);
    return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}
