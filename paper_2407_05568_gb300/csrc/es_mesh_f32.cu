// es_mesh_f32.cu -- the time step and the mesh redistribution of the mixed form on
// the FP32 pipe.
//
// The mixed form keeps the mesh as an FP32 displacement d = x - (x_00 + i dxi_1,
// y_00 + j dxi_2) from the Cartesian mesh (the stage kernels read it).  Here the
// CFL time step (eq. cfl), the monitor with G (eq. van der Waalsmonitor, or the
// smooth-test monitor), the low-pass filter, the Jacobi sweeps, the limiter
// Delta_gamma and the mesh velocity (Sec. 4) run on d in FP32: the Cartesian part
// of x is linear in the node index, so a neighbour's coordinate is its
// displacement plus +-dxi_k along its own direction, and its 6th-order difference
// is exactly dxi_k e_k.  On GB300 FP64 issues at 1/64 of the FP32 rate, and
// these kernels were a third of the mixed step at 200 x 200 in FP64.
#include <cuda_runtime.h>

#include "es_aux.h"
#include "es_bits.cuh"
#include "es_device.cuh"
#include "es_mesh_f32.h"

namespace es {

namespace {

__device__ __forceinline__ float block_max_f32(float v) {
    __shared__ float sh[32];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0f;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}

// the block maxima of four values in one pass (two barriers instead of eight)
__device__ __forceinline__ void block_max4_f32(float& a, float& b, float& c, float& d) {
    __shared__ float sh[4][32];
    for (int o = 16; o > 0; o >>= 1) {
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        c = fmaxf(c, __shfl_xor_sync(0xffffffffu, c, o));
        d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
        sh[2][w] = c;
        sh[3][w] = d;
    }
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    a = lane < nw ? sh[0][lane] : 0.0f;
    b = lane < nw ? sh[1][lane] : 0.0f;
    c = lane < nw ? sh[2][lane] : 0.0f;
    d = lane < nw ? sh[3][lane] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) {
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        c = fmaxf(c, __shfl_xor_sync(0xffffffffu, c, o));
        d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
    }
    __syncthreads();
}

__device__ __forceinline__ float block_min_f32(float v) {
    __shared__ float sh[32];
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = threadIdx.x < nw ? sh[threadIdx.x] : 3.0e38f;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}

// omega's coefficients alpha_k / max_k of the three monitor terms (0 where a maximum is 0), as floats: k_mon_f's
// last block forms them once (an FP64 division occupies the FP64 pipe, 1/64 of the FP32 rate on this GPU, for a
// whole warp whatever its active lanes; formed per warp they bounded the filter kernel)
__device__ __forceinline__ void set_mon_coeffs(DevScalars* d, const MonitorParams& mp) {
    const double M[3] = {__longlong_as_double((long long)atomicAdd(&d->red[RED_MON0], 0ULL)),
                         __longlong_as_double((long long)atomicAdd(&d->red[RED_MON1], 0ULL)),
                         __longlong_as_double((long long)atomicAdd(&d->red[RED_MON2], 0ULL))};
    const double w[3] = {mp.w0, mp.w1, mp.w2};
    for (int k = 0; k < 3; ++k) d->mon_c[k] = M[k] > 0.0 ? float(w[k] / M[k]) : 0.0f;
}

// a displacement ghost along one direction as at most two mesh nodes: periodic wrap (d is periodic),
// outflow odd reflection d_{-m} = 2 d_0 - d_m (the reflection of x, whose Cartesian part cancels); the
// mirror index is clamped to the mesh, as in ghost_terms.  Float weights (1, 2, -1, and their products,
// are exact), so the boundary nodes cost no FP64 work.
struct GhostF {
    int i0, i1;
    float w0, w1;
    bool two;
};

__device__ __forceinline__ GhostF ghost_f(int i, int n, int bc) {
    GhostF t;
    t.two = false;
    t.w0 = 1.0f;
    t.w1 = 0.0f;
    t.i1 = 0;
    if (i >= 0 && i < n) {
        t.i0 = i;
    } else if (bc == ES_BC_PERIODIC) {
        t.i0 = wrap_index(i, n);
    } else {
        int m = i < 0 ? -i : 2 * (n - 1) - i;
        m = m < 0 ? 0 : (m > n - 1 ? n - 1 : m);
        t.i0 = i < 0 ? 0 : n - 1;
        t.i1 = m;
        t.w0 = 2.0f;
        t.w1 = -1.0f;
        t.two = true;
    }
    return t;
}

// displacement at a ghost node (out of line: inlined at every neighbour read it made the per-node kernels' code long
// and branchy, and one-node-per-thread warps stall on instruction fetch; only boundary nodes call it)
__device__ __noinline__ float disp_ghost(int n1, int n2, int dim, int bc0, int bc1, const float* dc, int gi, int gj) {
    const GhostF ti = ghost_f(gi, n1, bc0);
    GhostF tj;
    if (dim == 2) {
        tj = ghost_f(gj, n2, bc1);
    } else {
        tj.i0 = 0; tj.i1 = 0; tj.w0 = 1.0f; tj.w1 = 0.0f; tj.two = false;
    }
    const size_t r0 = size_t(tj.i0) * n1, r1 = size_t(tj.i1) * n1;
    float acc = (ti.w0 * tj.w0) * dc[r0 + ti.i0];             // the terms in ghost_terms' order
    if (tj.two) acc += (ti.w0 * tj.w1) * dc[r1 + ti.i0];
    if (ti.two) {
        acc += (ti.w1 * tj.w0) * dc[r0 + ti.i1];
        if (tj.two) acc += (ti.w1 * tj.w1) * dc[r1 + ti.i1];
    }
    return acc;
}

// displacement at a node that may be a ghost
__device__ __forceinline__ float disp_at(const GridParams& g, const float* d, int gi, int gj, int comp) {
    const size_t N = size_t(g.n1) * g.n2;
    const float* dc = d + comp * N;
    if (gi >= 0 && gi < g.n1 && (g.dim == 1 || (gj >= 0 && gj < g.n2)))
        return dc[size_t(g.dim == 2 ? gj : 0) * g.n1 + gi];
    return disp_ghost(g.n1, g.n2, g.dim, g.bc[0], g.bc[1], dc, gi, gj);
}

__device__ __forceinline__ float field_at_f(const GridParams& g, const float* f, int i, int j) {
    const int si = state_index(i, g.n1, g.bc[0]);
    const int sj = g.dim == 2 ? state_index(j, g.n2, g.bc[1]) : 0;
    return f[sj * g.n1 + si];
}

// d x_comp / d xi_k at (i, j) from the 6th-order central difference of the displacement
__device__ __forceinline__ float dx_dxi(const GridParams& g, const float* d, int i, int j, int comp, int k,
                                        float inv_dxi) {
    float s = 0.0f;
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
        const float h = 0.5f * float(ec_alpha(m));
        if (k == 0) s += h * (disp_at(g, d, i + m, j, comp) - disp_at(g, d, i - m, j, comp));
        else s += h * (disp_at(g, d, i, j + m, comp) - disp_at(g, d, i, j - m, comp));
    }
    return (comp == k ? 1.0f : 0.0f) + s * inv_dxi;
}

// value of a mixed-form state entry: hi plane + lo plane
__device__ __forceinline__ float ld2(const float* a, size_t plane, size_t i) { return a[i] + a[plane + i]; }

__device__ __forceinline__ bool fixed_node_f(const GridParams& g, int i, int j) {
    bool f = g.bc[0] == ES_BC_OUTFLOW && (i == 0 || i == g.n1 - 1);
    if (g.dim == 2) f = f || (g.bc[1] == ES_BC_OUTFLOW && (j == 0 || j == g.n2 - 1));
    return f;
}

// the node term of eq. cfl on the FP32 pipe: sum_k (|J xi_{k,t} + n_k . v| + |n_k| c) / (J dxi_k) with
// J xi_{k,t} = -xdot . n_k, at node id with mesh velocity (xd1, xd2); a node without a real sound speed
// gives 3e38 (the time step then collapses and the admissibility check reports the state)
__device__ __forceinline__ float cfl_node_f(const GridParams& g, const GasF32& G, const float* JU, const float* J,
                                            const float* disp, int id, float xd1, float xd2, float* t0 = nullptr,
                                            float* t1 = nullptr) {
    const int N = g.n1 * g.n2;
    const size_t P = size_t(g.dim + 2) * N;
    const float idx1 = g.finv[0], idx2 = g.finv[1];
    const int i = id % g.n1, j = id / g.n1;
    const float iJ = 1.0f / ld2(J, N, id);
    const float rho = ld2(JU, P, id) * iJ;
    const float irho = 1.0f / rho;
    const float v1 = ld2(JU, P, N + id) * iJ * irho;
    const float v2 = g.dim == 2 ? ld2(JU, P, 2 * N + id) * iJ * irho : 0.0f;
    const float E = ld2(JU, P, (g.dim + 1) * N + id) * iJ;
    const float T = (E * irho - 0.5f * (v1 * v1 + v2 * v2) + G.a * rho) * G.icv;
    const float iom = 1.0f / (1.0f - G.b * rho);
    const float c2 = (1.0f + G.delta) * G.R * T * iom * iom - 2.0f * G.a * rho;
    const float c = sqrtf(fmaxf(c2, 0.0f));
    const bool ok = c2 > 0.0f;
    float tot;
    if (g.dim == 1) {
        tot = (fabsf(v1 - xd1) + c) * iJ * idx1;
        if (t0) {                                  // the terms of cfl_moving_term
            const float f = iJ * idx1;
            t0[id] = v1 * f;
            t0[N + id] = f;
            t0[2 * N + id] = ok ? c * f : 3.0e38f;
        }
    } else {
        float x1, x2, y1, y2;
        if (i >= 3 && i < g.n1 - 3 && j >= 3 && j < g.n2 - 3) {
            // interior: the 24 displacement loads have no ghost rule and are issued together
            float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};      // d x/d xi_1, d x/d xi_2, d y/d xi_1, d y/d xi_2
#pragma unroll
            for (int m = 1; m <= 3; ++m) {
                const float h = 0.5f * float(ec_alpha(m));
                s[0] += h * (disp[id + m] - disp[id - m]);
                s[1] += h * (disp[id + m * g.n1] - disp[id - m * g.n1]);
                s[2] += h * (disp[N + id + m] - disp[N + id - m]);
                s[3] += h * (disp[N + id + m * g.n1] - disp[N + id - m * g.n1]);
            }
            x1 = 1.0f + s[0] * idx1;
            x2 = s[1] * idx2;
            y1 = s[2] * idx1;
            y2 = 1.0f + s[3] * idx2;
        } else {
            x1 = dx_dxi(g, disp, i, j, 0, 0, idx1);
            x2 = dx_dxi(g, disp, i, j, 0, 1, idx2);
            y1 = dx_dxi(g, disp, i, j, 1, 0, idx1);
            y2 = dx_dxi(g, disp, i, j, 1, 1, idx2);
        }
        const float a1 = y2, b1 = -x2;        // J dxi_1/dx
        const float a2 = -y1, b2 = x1;        // J dxi_2/dx
        const float n1c = sqrtf(a1 * a1 + b1 * b1) * c, n2c = sqrtf(a2 * a2 + b2 * b2) * c;
        tot = (fabsf(a1 * (v1 - xd1) + b1 * (v2 - xd2)) + n1c) * iJ * idx1 +
              (fabsf(a2 * (v1 - xd1) + b2 * (v2 - xd2)) + n2c) * iJ * idx2;
        if (t0) {                                  // the terms of cfl_moving_term
            const float f1 = iJ * idx1, f2 = iJ * idx2;
            t0[id] = (a1 * v1 + b1 * v2) * f1;
            t0[N + id] = a1 * f1;
            t0[2 * N + id] = b1 * f1;
            t0[3 * N + id] = ok ? n1c * f1 : 3.0e38f;
            t1[id] = (a2 * v1 + b2 * v2) * f2;
            t1[N + id] = a2 * f2;
            t1[2 * N + id] = b2 * f2;
            t1[3 * N + id] = ok ? n2c * f2 : 0.0f;
        }
    }
    if (!ok) tot = 3.0e38f;
    return tot;
}

}  // namespace

// eq. cfl on the FP32 pipe: the maximum over the nodes of cfl_node_f goes to d->red[slot]; vel = nullptr
// is a mesh at rest.
__global__ void k_cfl_f(GridParams g, GasF32 G, const float* JU, const float* J, const float* disp, const float* vel,
                        int slot, DevScalars* d) {
    const int N = g.n1 * g.n2;
    float m = 0.0f;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const float xd1 = vel != nullptr ? vel[id] : 0.0f;
        const float xd2 = vel != nullptr && g.dim == 2 ? vel[N + id] : 0.0f;
        m = fmaxf(m, cfl_node_f(g, G, JU, J, disp, id, xd1, xd2));
    }
    m = block_max_f32(m);
    if (threadIdx.x == 0) atomic_max_pos(&d->red[slot], double(m));
}

// density and G = nu^3 p_nunu|_s / (2 c^2) at a node from the (hi, lo) state planes, in double-float
// arithmetic (near the critical point p_nunu is a difference of nearly equal terms: the EOS stays at
// FP64-like accuracy there); the monitor's differences of neighbours are formed from these pairs
__device__ __forceinline__ void mon_field_df(const GridParams& g, const GasF32& G, const float* JU, const float* J,
                                             int N, size_t P, int id, mixed::df* rho_out, mixed::df* G_out) {
    using mixed::df;
    df mom[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll
    for (int k = 0; k < 3; ++k)                    // fixed bound: the array stays in registers
        if (k < g.dim) mom[k] = {JU[(1 + k) * N + id], JU[P + (1 + k) * N + id]};
    const int ce = (g.dim + 1) * N + id;
    mixed::rho_G_df2({JU[id], JU[P + id]}, mom, g.dim, {JU[ce], JU[P + ce]}, {J[id], J[N + id]}, G.gdf, rho_out,
                     G_out);
}

// density and G of every node as (hi, lo) float planes: rhoF and GF hold 2 N floats each, the low parts
// N floats after the high parts
__global__ void k_mon_fields_f(GridParams g, GasF32 G, const float* JU, const float* J, float* rhoF, float* GF) {
    const int N = g.n1 * g.n2;
    const size_t P = size_t(g.dim + 2) * N;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        mixed::df r, G0;
        mon_field_df(g, G, JU, J, N, P, id, &r, &G0);
        rhoF[id] = r.hi;
        rhoF[N + id] = r.lo;
        GF[id] = G0.hi;
        GF[N + id] = G0.lo;
    }
}

// the monitor terms in one pass over TX x TY tiles (TX TY x 1 in 1D): the density and G of the tile's nodes and
// of a one-node halo (ghost rule of the state) are computed once each in double-float and kept in shared memory,
// then every node forms its differences from them.  With do_dt, thread 0 also sets the step's dt from the CFL
// maximum (k_dt's work: the CFL kernel has finished when this one starts).  MON_NT threads: 32 x 8 tiles take two
// rounds of the EOS per thread (1.33 evaluations per node), 30 x 6 tiles one (the tile with its halo is one node
// per thread, 1.42 evaluations per node): the first for throughput on large meshes, the second for latency on
// small ones.
template <int TX, int TY>
__global__ void __launch_bounds__(MON_NT, 4) k_mon_f(GridParams g, GasF32 G, const float* JU, const float* J,
                                                     MonitorParams mp, float* t0, float* t1, float* t2, DevScalars* d,
                                                     int do_dt, double cfl, double dt_fixed, const float* disp,
                                                     float* cfl_terms) {
    constexpr int CAP = (TX + 2) * (TY + 2);              // >= TX * TY + 2, the 1D tile with its halo
    static_assert(TX * TY <= MON_NT && CAP >= TX * TY + 2, "tile");
    __shared__ float srh[CAP], srl[CAP], sgh[CAP], sgl[CAP];
    if (do_dt == 1 && blockIdx.x == 0 && threadIdx.x == 0) set_dt_from_cfl(d, cfl, dt_fixed);
    const int N = g.n1 * g.n2;
    const size_t P = size_t(g.dim + 2) * N;
    const int TW = g.dim == 2 ? TX : TX * TY;            // tile width; 1D tiles are one row
    const int HW = TW + 2;
    const int ntx = (g.n1 + TW - 1) / TW;
    const int i0 = (blockIdx.x % ntx) * TW;
    const int j0 = g.dim == 2 ? (blockIdx.x / ntx) * TY : 0;
    const int hh = g.dim == 2 ? TY + 2 : 1;
    for (int t = threadIdx.x; t < HW * hh; t += blockDim.x) {
        const int lx = t % HW, ly = t / HW;
        const int gi = i0 - 1 + lx, gj = g.dim == 2 ? j0 - 1 + ly : 0;
        const int sidx = (g.dim == 2 ? state_index(gj, g.n2, g.bc[1]) : 0) * g.n1 + state_index(gi, g.n1, g.bc[0]);
        mixed::df r, Gv;
        mon_field_df(g, G, JU, J, N, P, sidx, &r, &Gv);
        srh[t] = r.hi;
        srl[t] = r.lo;
        sgh[t] = Gv.hi;
        sgl[t] = Gv.lo;
    }
    __syncthreads();
    float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f, mc = 0.0f;
    const int tx = threadIdx.x % TW, ty = threadIdx.x / TW;
    const int i = i0 + tx, j = j0 + ty;
    const bool owner = threadIdx.x < TW * (g.dim == 2 ? TY : 1);   // the others formed halo values only
    if (owner && i < g.n1 && (g.dim == 1 || j < g.n2)) {
        const int id = j * g.n1 + i;
        // do_dt == 2: eq. cfl with the mesh at rest at this node (k_cfl_f's work), and its terms for the moving pass
        if (do_dt == 2)
            mc = cfl_node_f(g, G, JU, J, disp, id, 0.0f, 0.0f, cfl_terms,
                            cfl_terms ? cfl_terms + 4 * size_t(N) : nullptr);
        const int c = (g.dim == 2 ? ty + 1 : 0) * HW + tx + 1;
        const mixed::df r0 = {srh[c], srl[c]}, G0 = {sgh[c], sgl[c]};
        float gr = 0.0f, gg = 0.0f, lg = 0.0f, lr = 0.0f;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (k >= g.dim) break;
            const float h = g.finv[k];
            const int off = k == 0 ? 1 : HW;
            const mixed::df rp = {srh[c + off], srl[c + off]}, Gp = {sgh[c + off], sgl[c + off]};
            const mixed::df rm = {srh[c - off], srl[c - off]}, Gm = {sgh[c - off], sgl[c - off]};
            const float a = mixed::df_diff(rp, rm) * 0.5f * h, b = mixed::df_diff(Gp, Gm) * 0.5f * h;
            const float cc = mixed::df_second_diff(Gp, G0, Gm) * h * h, e = mixed::df_second_diff(rp, r0, rm) * h * h;
            gr += a * a;
            gg += b * b;
            lg += cc * cc;
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
        m0 = v0;
        m1 = v1;
        m2 = v2;
    }
    block_max4_f32(m0, m1, m2, mc);                          // mc stays 0 unless do_dt == 2
    if (threadIdx.x == 0) {
        atomic_max_pos(&d->red[RED_MON0], double(m0));
        atomic_max_pos(&d->red[RED_MON1], double(m1));
        atomic_max_pos(&d->red[RED_MON2], double(m2));
        if (do_dt == 2) atomic_max_pos(&d->red[RED_CFL], double(mc));
        __threadfence();
        const unsigned int ticket = atomicAdd(&d->done, 1u);
        if (ticket == gridDim.x - 1) {                      // every block's maxima are in
            set_mon_coeffs(d, mp);
            if (do_dt == 2)                                 // the step's dt once every node is in
                set_dt_from_max(d, __longlong_as_double((long long)atomicAdd(&d->red[RED_CFL], 0ULL)), cfl, dt_fixed);
            d->done = 0u;
        }
    }
}

template <int TX, int TY>
static int mon_f_blocks(const GridParams& g) {
    if (g.dim == 1) return (g.n1 + TX * TY - 1) / (TX * TY);
    return ((g.n1 + TX - 1) / TX) * ((g.n2 + TY - 1) / TY);
}

void launch_mon_f(const GridParams& g, const GasF32& G, const float* JU, const float* J, const MonitorParams& mp,
                  float* t0, float* t1, float* t2, DevScalars* d, int do_dt, double cfl, double dt_fixed,
                  const float* disp, float* cfl_terms, int nsm, cudaStream_t s) {
    const int big = mon_f_blocks<32, 8>(g);
    if (big >= 4 * nsm)         // four resident CTAs per SM: at least one full wave
        k_mon_f<32, 8><<<big, MON_NT, 0, s>>>(g, G, JU, J, mp, t0, t1, t2, d, do_dt, cfl, dt_fixed, disp, cfl_terms);
    else
        k_mon_f<30, 6><<<mon_f_blocks<30, 6>(g), MON_NT, 0, s>>>(g, G, JU, J, mp, t0, t1, t2, d, do_dt, cfl, dt_fixed,
                                                                   disp, cfl_terms);
}


__global__ void k_mon_omega_f(GridParams g, MonitorParams mp, const float* t0, const float* t1, const float* t2,
                              const DevScalars* d, float* omega) {
    const int N = g.n1 * g.n2;
    // the coefficients from the maxima once per block (the 3D form's terms kernel leaves no float copies)
    __shared__ float cs[3];
    if (threadIdx.x == 0) {
        const double M0 = __longlong_as_double((long long)d->red[RED_MON0]);
        const double M1 = __longlong_as_double((long long)d->red[RED_MON1]);
        const double M2 = __longlong_as_double((long long)d->red[RED_MON2]);
        cs[0] = M0 > 0.0 ? float(mp.w0 / M0) : 0.0f;
        cs[1] = M1 > 0.0 ? float(mp.w1 / M1) : 0.0f;
        cs[2] = M2 > 0.0 ? float(mp.w2 / M2) : 0.0f;
    }
    __syncthreads();
    const float c0 = cs[0], c1 = cs[1], c2 = cs[2];
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x)
        omega[id] = sqrtf(1.0f + c0 * t0[id] + c1 * t1[id] + c2 * t2[id]);
}

// low-pass filter: omega_i <- sum_{j in {0,+-1}^d} (1/2)^(|j|_1 + d) omega_{i+j}
__global__ void k_filter_f(GridParams g, const float* in, float* out) {
    const int N = g.n1 * g.n2;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        float s;
        if (g.dim == 1) {
            s = 0.25f * field_at_f(g, in, i - 1, 0) + 0.5f * in[id] + 0.25f * field_at_f(g, in, i + 1, 0);
        } else {
            s = 0.0f;
            for (int dj = -1; dj <= 1; ++dj) {
                float row = 0.0f;
                for (int di = -1; di <= 1; ++di) row += (di == 0 ? 0.5f : 0.25f) * field_at_f(g, in, i + di, j + dj);
                s += (dj == 0 ? 0.5f : 0.25f) * row;
            }
        }
        out[id] = s;
    }
}

// Jacobi sweep k on the displacement: sweep 0 reads d and writes buf[0]; sweep k reads
// buf[(k-1)%2] and writes buf[k%2].  The coordinate of a neighbour along direction kk is
// its displacement plus +-dxi_kk in component kk.  Tolerance check as in the FP64 path.
__global__ void k_jacobi_f(GridParams g, const float* omega, const float* d0, float* da, float* db, int k,
                           DevScalars* d, int check, double eps) {
    if (d->conv) return;
    const int N = g.n1 * g.n2;
    const float* xin = k == 0 ? d0 : ((k - 1) & 1 ? db : da);
    float* xout = (k & 1) ? db : da;
    float chg = 0.0f;
    const float ih2k[2] = {g.finv2[0], g.finv2[1]};
    const float dxk[2] = {g.fdx[0], g.fdx[1]};
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        if (fixed_node_f(g, i, j)) {
            for (int c = 0; c < g.dim; ++c) xout[c * N + id] = xin[c * N + id];
            continue;
        }
        const float w0 = omega[id];
        float den = 0.0f, num0 = 0.0f, num1 = 0.0f;
        for (int kk = 0; kk < g.dim; ++kk) {
            const int di = kk == 0, dj = kk == 1;
            const float ih2 = kk == 0 ? ih2k[0] : ih2k[1];
            const float dx = kk == 0 ? dxk[0] : dxk[1];
            const float wp = 0.5f * (w0 + field_at_f(g, omega, i + di, j + dj)) * ih2;
            const float wm = 0.5f * (w0 + field_at_f(g, omega, i - di, j - dj)) * ih2;
            den += wp + wm;
            const float sp = kk == 0 ? dx : 0.0f, sp1 = kk == 1 ? dx : 0.0f;
            num0 += wp * (disp_at(g, xin, i + di, j + dj, 0) + sp) + wm * (disp_at(g, xin, i - di, j - dj, 0) - sp);
            if (g.dim == 2)
                num1 += wp * (disp_at(g, xin, i + di, j + dj, 1) + sp1) +
                        wm * (disp_at(g, xin, i - di, j - dj, 1) - sp1);
        }
        const float idn = 1.0f / den;
        const float n0 = num0 * idn;
        chg = fmaxf(chg, fabsf(n0 - xin[id]));
        xout[id] = n0;
        if (g.dim == 2) {
            const float n1 = num1 * idn;
            chg = fmaxf(chg, fabsf(n1 - xin[N + id]));
            xout[N + id] = n1;
        }
    }
    if (check) {
        chg = block_max_f32(chg);
        if (threadIdx.x == 0) {
            atomic_max_pos(&d->red[RED_JAC], double(chg));
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

__device__ __forceinline__ const float* jacobi_result_f(const DevScalars* d, const float* d0, const float* da,
                                                        const float* db) {
    if (d->sweeps == 0) return d0;
    return ((d->sweeps - 1) & 1) ? db : da;
}

// Delta_gamma on the displacement: the spacing to a neighbour along k is dxi_k + d_i - d_{i-1}
__global__ void k_limiter_f(GridParams g, const float* d0, const float* da, const float* db, DevScalars* d) {
    const int N = g.n1 * g.n2;
    const float* xit = jacobi_result_f(d, d0, da, db);
    float m = 1.0f;
    const float hk[2] = {g.fdx[0], g.fdx[1]};
#pragma unroll 4
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int i = id % g.n1, j = id / g.n1;
        for (int k = 0; k < g.dim; ++k) {
            const float dx = xit[k * N + id] - d0[k * N + id];
            const int di = k == 0, dj = k == 1;
            const float h = k == 0 ? hk[0] : hk[1];
            if (dx < 0.0f) m = fminf(m, -(h + d0[k * N + id] - disp_at(g, d0, i - di, j - dj, k)) / (2.0f * dx));
            else if (dx > 0.0f) m = fminf(m, (h + disp_at(g, d0, i + di, j + dj, k) - d0[k * N + id]) / (2.0f * dx));
        }
    }
    m = block_min_f32(m);
    if (threadIdx.x == 0) atomic_min_pos(&d->red[RED_GAMMA], double(m));
}

// xdot = Delta_gamma (x^[mu] - x^n) / dt: float (for the stage kernels) and double (the API's array).
// cfl > 0 also takes eq. cfl with this mesh velocity at each node from the terms the mesh-at-rest CFL pass
// stored (cfl_moving_term), and the last block to finish shrinks the step's dt to it (k_dt_moving's work).
__global__ void k_velocity_f(GridParams g, const float* __restrict__ d0, const float* __restrict__ da,
                             const float* __restrict__ db, DevScalars* d, float* __restrict__ fxd,
                             double* __restrict__ xdot, const float* __restrict__ terms, double cfl) {
    const int N = g.n1 * g.n2;
    const float* xit = jacobi_result_f(d, d0, da, db);
    __shared__ float fs;                // Delta_gamma / dt, formed once per block (FP64 division)
    if (threadIdx.x == 0) {
        const double gam = __longlong_as_double((long long)d->red[RED_GAMMA]);
        const double dt = d->dt;
        fs = dt > 0.0 ? float(gam / dt) : 0.0f;
    }
    __syncthreads();
    const float f = fs;
    const bool moving_cfl = cfl > 0.0;  // compared once, not per node (an FP64 comparison)
    float m = 0.0f;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const float v1 = f * (xit[id] - d0[id]);
        fxd[id] = v1;
        xdot[id] = bits::widen(v1);
        float v2 = 0.0f;
        if (g.dim == 2) {
            v2 = f * (xit[N + id] - d0[N + id]);
            fxd[N + id] = v2;
            xdot[N + id] = bits::widen(v2);
        }
        if (moving_cfl) m = fmaxf(m, cfl_moving_term(terms, terms + 4 * size_t(N), size_t(N), size_t(id), g.dim, v1, v2));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d->gamma = __longlong_as_double((long long)d->red[RED_GAMMA]);
        d->sweeps_total += d->sweeps;
        d->solves += 1;
    }
    if (cfl > 0.0) {
        m = block_max_f32(m);
        if (threadIdx.x == 0) {
            atomic_max_pos(&d->red[RED_CFL2], double(m));
            __threadfence();
            const unsigned int ticket = atomicAdd(&d->done, 1u);
            if (ticket == gridDim.x - 1) {          // every block's maximum is in: every block has read dt
                shrink_dt_to(d, __longlong_as_double((long long)atomicAdd(&d->red[RED_CFL2], 0ULL)), cfl);
                d->done = 0u;
            }
        }
    }
}

}  // namespace es

namespace es {

// ---------------------------------------------------------------- fused passes (2D)
// omega with s filter passes, and mu Jacobi sweeps without a tolerance, each in one launch, on register
// tiles.  A CTA owns a tile RT_W = 64 nodes wide and NW x RW tall, halo included; lane L of warp w keeps
// columns 2L and 2L+1 of the warp's band of RW rows in registers.  A node's horizontal neighbours are in its
// own lane or the adjacent one (one shuffle each), its vertical ones in the lane's registers, and the rows
// just outside a band are the neighbouring warps' edge rows, exchanged through shared memory once per pass
// (one barrier).  After p passes the p outermost columns and rows of the tile are stale, so a tile's output
// is the tile less a band of h = s (or mu) nodes; periodic halos hold the wrapped nodes and evolve with them.
// At an outflow end the filter reads the end node in place of its missing neighbour (the unfused kernels'
// clamped index), and the sweeps leave the end nodes where they are, so neither reads beyond the mesh.  The
// arithmetic per node is that of k_mon_omega_f, k_filter_f and k_jacobi_f, in the same order.
constexpr int RT_W = 64;           // halos up to 8 nodes (the callers pass 1 .. 8 passes or sweeps)

// the left neighbour of column 2L (lane L-1's column 2L+1) and the right neighbour of column 2L+1 (lane
// L+1's column 2L); lanes 0 and 31 get their own value back: the tile's edge columns, never output
__device__ __forceinline__ float from_left(float b) { return __shfl_up_sync(0xffffffffu, b, 1); }
__device__ __forceinline__ float from_right(float a) { return __shfl_down_sync(0xffffffffu, a, 1); }

// one 1/4 1/2 1/4 row of the filter, summed as k_filter_f sums it
__device__ __forceinline__ float filter3(float l, float c, float r) {
    float s = 0.0f;
    s += 0.25f * l;
    s += 0.5f * c;
    s += 0.25f * r;
    return s;
}

// the filter's row sums at columns a = 2L and b = 2L+1; CX: outflow ends along xi_1, where the end node
// stands in for its missing neighbour
struct EndCols {
    bool a_first, a_last, b_first, b_last;
};

template <bool CX>
__device__ __forceinline__ void filter_row(float a, float b, const EndCols& e, float& ra, float& rb) {
    float la = from_left(b), rgt_a = b, lb = a, rgt_b = from_right(a);
    if (CX) {
        if (e.a_first) la = a;
        if (e.a_last) rgt_a = a;
        if (e.b_first) lb = b;
        if (e.b_last) rgt_b = b;
    }
    ra = filter3(la, a, rgt_a);
    rb = filter3(lb, b, rgt_b);
}

// the passes of one warp's band (va, vb: columns 2L and 2L+1); CY: outflow ends along xi_2, yb: the band's
// first mesh row
template <int NW, int RW, bool CX, bool CY>
__device__ __forceinline__ void filter_passes(float (&va)[RW], float (&vb)[RW], float (*edge)[NW][2][RT_W], int h,
                                              int w, int lane, int yb, int n2, const EndCols& e) {
    for (int p = 0; p < h; ++p) {
        float(*E)[2][RT_W] = edge[p & 1];
        *reinterpret_cast<float2*>(&E[w][0][2 * lane]) = make_float2(va[0], vb[0]);
        *reinterpret_cast<float2*>(&E[w][1][2 * lane]) = make_float2(va[RW - 1], vb[RW - 1]);
        __syncthreads();
        // the rows above and below the band (the tile's first and last warps: their own edge rows, stale)
        const float2 up = w > 0 ? *reinterpret_cast<const float2*>(&E[w - 1][1][2 * lane]) : make_float2(va[0], vb[0]);
        const float2 dn = w < NW - 1 ? *reinterpret_cast<const float2*>(&E[w + 1][0][2 * lane])
                                     : make_float2(va[RW - 1], vb[RW - 1]);
        float ra[RW + 2], rb[RW + 2];
        filter_row<CX>(up.x, up.y, e, ra[0], rb[0]);
#pragma unroll
        for (int r = 0; r < RW; ++r) filter_row<CX>(va[r], vb[r], e, ra[r + 1], rb[r + 1]);
        filter_row<CX>(dn.x, dn.y, e, ra[RW + 1], rb[RW + 1]);
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            float ua = ra[r], ub = rb[r], da = ra[r + 2], db = rb[r + 2];
            if (CY) {
                if (yb + r == 0) {
                    ua = ra[r + 1];
                    ub = rb[r + 1];
                }
                if (yb + r == n2 - 1) {
                    da = ra[r + 1];
                    db = rb[r + 1];
                }
            }
            va[r] = filter3(ua, ra[r + 1], da);
            vb[r] = filter3(ub, rb[r + 1], db);
        }
    }
}

template <int NW, int RW>
__global__ void __launch_bounds__(NW * 32) k_omega_filter_r(GridParams g, MonitorParams mp,
                                                            const float* __restrict__ t0,
                                                            const float* __restrict__ t1,
                                                            const float* __restrict__ t2, const DevScalars* d,
                                                            int h, float* __restrict__ out) {
    __shared__ __align__(16) float edge[2][NW][2][RT_W];         // [pass parity][warp][first / last row][column]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int OX = RT_W - 2 * h, OY = NW * RW - 2 * h;
    const int x0 = blockIdx.x * OX - h, y0 = blockIdx.y * OY - h;
    const int xa = x0 + 2 * lane, yb = y0 + w * RW;
    const float c0 = d->mon_c[0], c1 = d->mon_c[1], c2 = d->mon_c[2];
    const int sa = state_index(xa, g.n1, g.bc[0]), sb = state_index(xa + 1, g.n1, g.bc[0]);
    float va[RW], vb[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const size_t row = size_t(state_index(yb + r, g.n2, g.bc[1])) * g.n1;
        va[r] = sqrtf(1.0f + c0 * t0[row + sa] + c1 * t1[row + sa] + c2 * t2[row + sa]);
        vb[r] = sqrtf(1.0f + c0 * t0[row + sb] + c1 * t1[row + sb] + c2 * t2[row + sb]);
    }
    const EndCols e = {xa == 0, xa == g.n1 - 1, xa + 1 == 0, xa + 1 == g.n1 - 1};
    // only tiles that reach an outflow end take the clamped reads
    const bool cx = g.bc[0] == ES_BC_OUTFLOW && (x0 <= 0 || x0 + RT_W >= g.n1);
    const bool cy = g.bc[1] == ES_BC_OUTFLOW && (y0 <= 0 || y0 + NW * RW >= g.n2);
    if (cx) {
        if (cy) filter_passes<NW, RW, true, true>(va, vb, edge, h, w, lane, yb, g.n2, e);
        else filter_passes<NW, RW, true, false>(va, vb, edge, h, w, lane, yb, g.n2, e);
    } else {
        if (cy) filter_passes<NW, RW, false, true>(va, vb, edge, h, w, lane, yb, g.n2, e);
        else filter_passes<NW, RW, false, false>(va, vb, edge, h, w, lane, yb, g.n2, e);
    }
    const bool ina = 2 * lane >= h && 2 * lane < h + OX && xa < g.n1;
    const bool inb = 2 * lane + 1 >= h && 2 * lane + 1 < h + OX && xa + 1 < g.n1;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int tr = w * RW + r;
        if (tr < h || tr >= h + OY || yb + r >= g.n2) continue;
        float* o = out + size_t(yb + r) * g.n1;
        if (ina) o[xa] = va[r];
        if (inb) o[xa + 1] = vb[r];
    }
}

// tiles NW x 4 rows tall: 64 rows (NW = 16) where the mesh gives at least four waves of them with per_sm
// resident CTAs per SM, else 32 (more CTAs at a larger share of halo)
constexpr int RT_RW = 4;

template <int NW>
static dim3 rt_grid(const GridParams& g, int h) {
    return dim3((g.n1 + RT_W - 2 * h - 1) / (RT_W - 2 * h), (g.n2 + NW * RT_RW - 2 * h - 1) / (NW * RT_RW - 2 * h));
}

static bool rt_tall(const GridParams& g, int h, int per_sm) {
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || n < 1)
            n = 1;
        nsm = n;
    }
    const dim3 t = rt_grid<16>(g, h);
    return size_t(t.x) * t.y >= size_t(4) * per_sm * nsm;
}

void launch_omega_filter(const GridParams& g, const MonitorParams& mp, const float* t0, const float* t1,
                         const float* t2, const DevScalars* d, int passes, float* out, cudaStream_t s) {
    if (rt_tall(g, passes, 3))
        k_omega_filter_r<16, RT_RW><<<rt_grid<16>(g, passes), 16 * 32, 0, s>>>(g, mp, t0, t1, t2, d, passes, out);
    else
        k_omega_filter_r<8, RT_RW><<<rt_grid<8>(g, passes), 8 * 32, 0, s>>>(g, mp, t0, t1, t2, d, passes, out);
}

// a node's sweep weights (constant over the sweeps), formed as k_jacobi_f forms them: the east face weight
// 0.5 (w_0 + w_E) / dxi_1^2, the north one likewise with dxi_2, and the reciprocal of the four faces' sum.  A
// node's west (south) face weight is its west (south) neighbour's east (north) one, the same float (the sum
// w_0 + w_W is commutative), so each face is formed once.
struct NodeW {
    float px, py, idn;
};

__device__ __forceinline__ NodeW node_weights(float w0, float we, float ww, float wn, float ws, float ih2x,
                                              float ih2y, float& mx, float& my) {
    NodeW n;
    float den = 0.0f;
    n.px = 0.5f * (w0 + we) * ih2x;
    mx = 0.5f * (w0 + ww) * ih2x;
    den += n.px + mx;
    n.py = 0.5f * (w0 + wn) * ih2y;
    my = 0.5f * (w0 + ws) * ih2y;
    den += n.py + my;
    n.idn = 1.0f / den;
    return n;
}

// one node's Jacobi update from its face weights (px, mx: east, west; py, my: north, south) and its
// neighbours' displacements (e, w, n, s; 0 and 1 the components), in k_jacobi_f's order (k_jacobi_f also adds
// +-0 to the neighbours' components across the other direction, which changes no value)
__device__ __forceinline__ void node_sweep(float px, float mx, float py, float my, float idn, float e0, float w0,
                                           float n0, float s0, float e1, float w1, float n1, float s1, float dxx,
                                           float dxy, float& o0, float& o1) {
    float num0 = px * (e0 + dxx) + mx * (w0 - dxx);
    float num1 = px * e1 + mx * w1;
    num0 += py * n0 + my * s0;
    num1 += py * (n1 + dxy) + my * (s1 - dxy);
    o0 = num0 * idn;
    o1 = num1 * idn;
}

// Delta_gamma's bound at one node and direction (k_limiter_f's rule): d0 the node's starting displacement,
// v its result, dm and dp the starting displacements of its neighbours before and after it, h the spacing
__device__ __forceinline__ float limit_term(float lim, float v, float d0, float dm, float dp, float h) {
    const float dx = v - d0;
    if (dx < 0.0f) lim = fminf(lim, -(h + d0 - dm) / (2.0f * dx));
    else if (dx > 0.0f) lim = fminf(lim, (h + dp - d0) / (2.0f * dx));
    return lim;
}

template <int NW, int RW>
__global__ void __launch_bounds__(NW * 32) k_jacobi_r(GridParams g, const float* __restrict__ omega,
                                                      const float* __restrict__ d0, float* __restrict__ dout, int h,
                                                      DevScalars* dv, int limit) {
    __shared__ __align__(16) float edge[2][NW][2][2][RT_W];      // [sweep parity][warp][first / last row][comp][col]
    __shared__ __align__(16) float start1[NW][2][RT_W];          // the starting xi_2 component of those rows
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int OX = RT_W - 2 * h, OY = NW * RW - 2 * h;
    const int x0 = blockIdx.x * OX - h, y0 = blockIdx.y * OY - h;
    const int xa = x0 + 2 * lane, yb = y0 + w * RW;
    const float ih2x = g.finv2[0], ih2y = g.finv2[1], dxx = g.fdx[0], dxy = g.fdx[1];
    // periodic halos hold the wrapped nodes (the displacement is periodic); an outflow ghost holds its clamped
    // node, which no moving node reads (the end nodes stay where they are)
    const int sa = state_index(xa, g.n1, g.bc[0]), sb = state_index(xa + 1, g.n1, g.bc[0]);
    const size_t N = size_t(g.n1) * g.n2;
    // the sweep weights from omega on the band and the rows above and below it
    NodeW qa[RW], qb[RW];
    float mxa[RW];                  // west face of column 2L (column 2L+1's west face is column 2L's east one)
    float mya0, myb0;               // south faces of the band's first row (the others: the row below's north)
    {
        float Wa[RW + 2], Wb[RW + 2];
#pragma unroll
        for (int r = 0; r < RW + 2; ++r) {
            const size_t row = size_t(state_index(yb + r - 1, g.n2, g.bc[1])) * g.n1;
            Wa[r] = omega[row + sa];
            Wb[r] = omega[row + sb];
        }
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const float a = Wa[r + 1], b = Wb[r + 1];
            float mx, mya, myb;
            qa[r] = node_weights(a, b, from_left(b), Wa[r + 2], Wa[r], ih2x, ih2y, mxa[r], mya);
            qb[r] = node_weights(b, from_right(a), a, Wb[r + 2], Wb[r], ih2x, ih2y, mx, myb);
            if (r == 0) {
                mya0 = mya;
                myb0 = myb;
            }
        }
    }
    float a0[RW], b0[RW], a1[RW], b1[RW];                         // displacement components at columns 2L, 2L+1
    float sa0[RW], sb0[RW], sa1[RW], sb1[RW];                     // their starting values (the limiter's)
    unsigned int moves = 0u;                                      // bit 2r: column 2L of row r, 2r+1: column 2L+1
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int gy = yb + r;
        const size_t row = size_t(state_index(gy, g.n2, g.bc[1])) * g.n1;
        a0[r] = sa0[r] = d0[row + sa];
        a1[r] = sa1[r] = d0[N + row + sa];
        b0[r] = sb0[r] = d0[row + sb];
        b1[r] = sb1[r] = d0[N + row + sb];
        const bool out_y = g.bc[1] == ES_BC_OUTFLOW && (gy < 0 || gy >= g.n2);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int gx = xa + c;
            const bool outside = out_y || (g.bc[0] == ES_BC_OUTFLOW && (gx < 0 || gx >= g.n1));
            if (!(outside || fixed_node_f(g, gx, gy))) moves |= 1u << (2 * r + c);
        }
    }
    if (limit) {
        *reinterpret_cast<float2*>(&start1[w][0][2 * lane]) = make_float2(sa1[0], sb1[0]);
        *reinterpret_cast<float2*>(&start1[w][1][2 * lane]) = make_float2(sa1[RW - 1], sb1[RW - 1]);
    }
    for (int p = 0; p < h; ++p) {
        float(*E)[2][2][RT_W] = edge[p & 1];
        *reinterpret_cast<float2*>(&E[w][0][0][2 * lane]) = make_float2(a0[0], b0[0]);
        *reinterpret_cast<float2*>(&E[w][0][1][2 * lane]) = make_float2(a1[0], b1[0]);
        *reinterpret_cast<float2*>(&E[w][1][0][2 * lane]) = make_float2(a0[RW - 1], b0[RW - 1]);
        *reinterpret_cast<float2*>(&E[w][1][1][2 * lane]) = make_float2(a1[RW - 1], b1[RW - 1]);
        __syncthreads();
        // rows above and below the band (the tile's first and last warps: their own edge rows, stale)
        const float2 u0 = w > 0 ? *reinterpret_cast<const float2*>(&E[w - 1][1][0][2 * lane]) : make_float2(a0[0], b0[0]);
        const float2 u1 = w > 0 ? *reinterpret_cast<const float2*>(&E[w - 1][1][1][2 * lane]) : make_float2(a1[0], b1[0]);
        const float2 l0 = w < NW - 1 ? *reinterpret_cast<const float2*>(&E[w + 1][0][0][2 * lane])
                                     : make_float2(a0[RW - 1], b0[RW - 1]);
        const float2 l1 = w < NW - 1 ? *reinterpret_cast<const float2*>(&E[w + 1][0][1][2 * lane])
                                     : make_float2(a1[RW - 1], b1[RW - 1]);
        float pa0 = u0.x, pb0 = u0.y, pa1 = u1.x, pb1 = u1.y;     // the old values of the row below row r
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const float ta0 = r < RW - 1 ? a0[r + 1] : l0.x, tb0 = r < RW - 1 ? b0[r + 1] : l0.y;
            const float ta1 = r < RW - 1 ? a1[r + 1] : l1.x, tb1 = r < RW - 1 ? b1[r + 1] : l1.y;
            const float mya = r > 0 ? qa[r - 1].py : mya0, myb = r > 0 ? qb[r - 1].py : myb0;
            float o0, o1, q0, q1;
            node_sweep(qa[r].px, mxa[r], qa[r].py, mya, qa[r].idn, b0[r], from_left(b0[r]), ta0, pa0, b1[r],
                       from_left(b1[r]), ta1, pa1, dxx, dxy, o0, o1);
            node_sweep(qb[r].px, qa[r].px, qb[r].py, myb, qb[r].idn, from_right(a0[r]), a0[r], tb0, pb0,
                       from_right(a1[r]), a1[r], tb1, pb1, dxx, dxy, q0, q1);
            pa0 = a0[r];
            pb0 = b0[r];
            pa1 = a1[r];
            pb1 = b1[r];
            if ((moves >> (2 * r)) & 1u) {
                a0[r] = o0;
                a1[r] = o1;
            }
            if ((moves >> (2 * r + 1)) & 1u) {
                b0[r] = q0;
                b1[r] = q1;
            }
        }
    }
    // output, and Delta_gamma from the starting values in registers: the xi_1 neighbours by shuffle, the xi_2
    // ones from the band or the neighbouring bands' edge rows (the tile's output nodes are at least one node
    // inside the tile, so every neighbour they read is a tile node; at an outflow end the end nodes do not move
    // and read none)
    if (limit) __syncthreads();
    float lim = 1.0f;                                        // limit: k_limiter_f's min over this tile's nodes
    const bool ina = 2 * lane >= h && 2 * lane < h + OX && xa < g.n1;
    const bool inb = 2 * lane + 1 >= h && 2 * lane + 1 < h + OX && xa + 1 < g.n1;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const float wa = from_left(sb0[r]), eb = from_right(sa0[r]);     // every lane shuffles
        const int tr = w * RW + r, gy = yb + r;
        if (tr < h || tr >= h + OY || gy >= g.n2) continue;
        const size_t row = size_t(gy) * g.n1;
        float sa1m, sb1m, sa1p, sb1p;                        // xi_2 neighbours' starting component 1
        if (r > 0) {
            sa1m = sa1[r - 1];
            sb1m = sb1[r - 1];
        } else {
            sa1m = start1[w - 1][1][2 * lane];
            sb1m = start1[w - 1][1][2 * lane + 1];
        }
        if (r < RW - 1) {
            sa1p = sa1[r + 1];
            sb1p = sb1[r + 1];
        } else {
            sa1p = start1[w + 1][0][2 * lane];
            sb1p = start1[w + 1][0][2 * lane + 1];
        }
        if (ina) {
            dout[row + xa] = a0[r];
            dout[N + row + xa] = a1[r];
            if (limit) {
                lim = limit_term(lim, a0[r], sa0[r], wa, sb0[r], dxx);
                lim = limit_term(lim, a1[r], sa1[r], sa1m, sa1p, dxy);
            }
        }
        if (inb) {
            dout[row + xa + 1] = b0[r];
            dout[N + row + xa + 1] = b1[r];
            if (limit) {
                lim = limit_term(lim, b0[r], sb0[r], sa0[r], eb, dxx);
                lim = limit_term(lim, b1[r], sb1[r], sb1m, sb1p, dxy);
            }
        }
    }
    if (limit) {
        lim = block_min_f32(lim);
        if (threadIdx.x == 0) atomic_min_pos(&dv->red[RED_GAMMA], double(lim));
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) atomicAdd(&dv->sweeps, h);
}

void launch_jacobi_tiles(const GridParams& g, const float* omega, const float* d0, float* dout, int sweeps,
                         DevScalars* dv, int limit, cudaStream_t s) {
    if (rt_tall(g, sweeps, 1))
        k_jacobi_r<16, RT_RW><<<rt_grid<16>(g, sweeps), 16 * 32, 0, s>>>(g, omega, d0, dout, sweeps, dv, limit);
    else
        k_jacobi_r<8, RT_RW><<<rt_grid<8>(g, sweeps), 8 * 32, 0, s>>>(g, omega, d0, dout, sweeps, dv, limit);
}

}  // namespace es
