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

// displacement at a node that may be a ghost
__device__ __forceinline__ float disp_at(const GridParams& g, const float* d, int gi, int gj, int comp) {
    const size_t N = size_t(g.n1) * g.n2;
    const float* dc = d + comp * N;
    if (gi >= 0 && gi < g.n1 && (g.dim == 1 || (gj >= 0 && gj < g.n2)))
        return dc[size_t(g.dim == 2 ? gj : 0) * g.n1 + gi];
    const GhostF ti = ghost_f(gi, g.n1, g.bc[0]);
    GhostF tj;
    if (g.dim == 2) {
        tj = ghost_f(gj, g.n2, g.bc[1]);
    } else {
        tj.i0 = 0; tj.i1 = 0; tj.w0 = 1.0f; tj.w1 = 0.0f; tj.two = false;
    }
    const size_t r0 = size_t(tj.i0) * g.n1, r1 = size_t(tj.i1) * g.n1;
    float acc = (ti.w0 * tj.w0) * dc[r0 + ti.i0];             // the terms in ghost_terms' order
    if (tj.two) acc += (ti.w0 * tj.w1) * dc[r1 + ti.i0];
    if (ti.two) {
        acc += (ti.w1 * tj.w0) * dc[r0 + ti.i1];
        if (tj.two) acc += (ti.w1 * tj.w1) * dc[r1 + ti.i1];
    }
    return acc;
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
    const float idx1 = float(g.inv_dxi[0]), idx2 = float(g.inv_dxi[1]);
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

// the monitor terms in one pass over MON_TX x MON_TY tiles (MON_TX x 1 in 1D): the density and G of the
// tile's nodes and of a one-node halo (ghost rule of the state) are computed once each in double-float and kept
// in shared memory, then every node forms its differences from them.  With do_dt, thread 0 also sets the step's
// dt from the CFL maximum (k_dt's work: the CFL kernel has finished when this one starts).
__global__ void __launch_bounds__(MON_TX * MON_TY) k_mon_f(GridParams g, GasF32 G, const float* JU, const float* J,
                                                           MonitorParams mp, float* t0, float* t1, float* t2,
                                                           DevScalars* d, int do_dt, double cfl, double dt_fixed,
                                                           const float* disp, float* cfl_terms) {
    constexpr int CAP = (MON_TX + 2) * (MON_TY + 2);      // >= MON_TX * MON_TY + 2, the 1D tile with its halo
    __shared__ float srh[CAP], srl[CAP], sgh[CAP], sgl[CAP];
    if (do_dt == 1 && blockIdx.x == 0 && threadIdx.x == 0) set_dt_from_cfl(d, cfl, dt_fixed);
    const int N = g.n1 * g.n2;
    const size_t P = size_t(g.dim + 2) * N;
    const int TW = g.dim == 2 ? MON_TX : MON_TX * MON_TY;  // tile width; 1D tiles are one row of all threads
    const int HW = TW + 2;
    const int ntx = (g.n1 + TW - 1) / TW;
    const int i0 = (blockIdx.x % ntx) * TW;
    const int j0 = g.dim == 2 ? (blockIdx.x / ntx) * MON_TY : 0;
    const int hh = g.dim == 2 ? MON_TY + 2 : 1;
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
    if (i < g.n1 && (g.dim == 1 || j < g.n2)) {
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
            const float h = float(g.inv_dxi[k]);
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
    m0 = block_max_f32(m0);
    m1 = block_max_f32(m1);
    m2 = block_max_f32(m2);
    if (threadIdx.x == 0) {
        atomic_max_pos(&d->red[RED_MON0], double(m0));
        atomic_max_pos(&d->red[RED_MON1], double(m1));
        atomic_max_pos(&d->red[RED_MON2], double(m2));
    }
    if (do_dt == 2) {                                        // uniform: the step's dt once every node is in
        mc = block_max_f32(mc);
        if (threadIdx.x == 0) {
            atomic_max_pos(&d->red[RED_CFL], double(mc));
            __threadfence();
            const unsigned int ticket = atomicAdd(&d->done, 1u);
            if (ticket == gridDim.x - 1) {
                set_dt_from_max(d, __longlong_as_double((long long)atomicAdd(&d->red[RED_CFL], 0ULL)), cfl, dt_fixed);
                d->done = 0u;
            }
        }
    }
}

int mon_f_blocks(const GridParams& g) {
    if (g.dim == 1) return (g.n1 + MON_TX * MON_TY - 1) / (MON_TX * MON_TY);
    return ((g.n1 + MON_TX - 1) / MON_TX) * ((g.n2 + MON_TY - 1) / MON_TY);
}


__global__ void k_mon_omega_f(GridParams g, MonitorParams mp, const float* t0, const float* t1, const float* t2,
                              const DevScalars* d, float* omega) {
    const int N = g.n1 * g.n2;
    const double M0 = __longlong_as_double((long long)d->red[RED_MON0]);
    const double M1 = __longlong_as_double((long long)d->red[RED_MON1]);
    const double M2 = __longlong_as_double((long long)d->red[RED_MON2]);
    const float c0 = M0 > 0.0 ? float(mp.w0 / M0) : 0.0f;
    const float c1 = M1 > 0.0 ? float(mp.w1 / M1) : 0.0f;
    const float c2 = M2 > 0.0 ? float(mp.w2 / M2) : 0.0f;
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
    const float ih2k[2] = {float(g.inv_dxi[0] * g.inv_dxi[0]), float(g.inv_dxi[1] * g.inv_dxi[1])};
    const float dxk[2] = {float(1.0 / g.inv_dxi[0]), float(1.0 / g.inv_dxi[1])};
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
    const float hk[2] = {float(1.0 / g.inv_dxi[0]), float(1.0 / g.inv_dxi[1])};
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
    const double gam = __longlong_as_double((long long)d->red[RED_GAMMA]);
    const double dt = d->dt;
    const float f = dt > 0.0 ? float(gam / dt) : 0.0f;
    float m = 0.0f;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const float v1 = f * (xit[id] - d0[id]);
        fxd[id] = v1;
        xdot[id] = double(v1);
        float v2 = 0.0f;
        if (g.dim == 2) {
            v2 = f * (xit[N + id] - d0[N + id]);
            fxd[N + id] = v2;
            xdot[N + id] = double(v2);
        }
        if (cfl > 0.0) m = fmaxf(m, cfl_moving_term(terms, terms + 4 * size_t(N), size_t(N), size_t(id), g.dim, v1, v2));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d->gamma = gam;
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
// omega + s filter passes, and mu Jacobi sweeps without a tolerance, each in one launch: a CTA
// owns a 32 x 16 tile and recomputes a halo of s (or mu) nodes in shared memory, so a pass
// needs no grid-wide step.  Ghost nodes follow the unfused kernels: periodic halos hold the
// wrapped nodes (and evolve with them); an outflow ghost of the filter is reset to its clamped
// boundary node after every pass; outflow boundary nodes of the mesh do not move, so the sweeps
// never read beyond them.  The arithmetic per node is that of k_mon_omega_f, k_filter_f and
// k_jacobi_f, in the same order.
constexpr int FT_X = 32, FT_Y = 16, FT_HMAX = 8;
constexpr int FT_W = FT_X + 2 * FT_HMAX, FT_H = FT_Y + 2 * FT_HMAX;

// the (x, y) cell of a TW-wide tile one block stride further on (the strided loops below step
// the cell without an integer division per iteration)
__device__ __forceinline__ void next_cell(int& sx, int& sy, int2 sq, int TW) {
    sx += sq.x;
    sy += sq.y;
    if (sx >= TW) {
        sx -= TW;
        ++sy;
    }
}

// (templated on the value type; the FP64 form keeps one pass per launch: in FP64 the halo
// recomputation costs more than the launches it saves)
template <class T>
__global__ void __launch_bounds__(256) k_omega_filter_t(GridParams g, MonitorParams mp, const T* t0, const T* t1,
                                                        const T* t2, const DevScalars* d, int passes, T* out) {
    __shared__ T A[FT_W * FT_H], B[FT_W * FT_H];
    const int h = passes, TW = FT_X + 2 * h, TH = FT_Y + 2 * h;
    const int2 sq = make_int2(int(blockDim.x) % TW, int(blockDim.x) / TW);   // one stride in cells
    const int x0 = blockIdx.x * FT_X - h, y0 = blockIdx.y * FT_Y - h;
    const double M0 = __longlong_as_double((long long)d->red[RED_MON0]);
    const double M1 = __longlong_as_double((long long)d->red[RED_MON1]);
    const double M2 = __longlong_as_double((long long)d->red[RED_MON2]);
    const T c0 = M0 > 0.0 ? T(mp.w0 / M0) : T(0);
    const T c1 = M1 > 0.0 ? T(mp.w1 / M1) : T(0);
    const T c2 = M2 > 0.0 ? T(mp.w2 / M2) : T(0);
    for (int idx = threadIdx.x, sx = idx % TW, sy = idx / TW; idx < TW * TH;
         idx += blockDim.x, next_cell(sx, sy, sq, TW)) {
        const int si = state_index(x0 + sx, g.n1, g.bc[0]), sj = state_index(y0 + sy, g.n2, g.bc[1]);
        const int id = sj * g.n1 + si;
        A[idx] = sqrt(T(1) + c0 * t0[id] + c1 * t1[id] + c2 * t2[id]);
    }
    __syncthreads();
    T* cur = A;
    T* nxt = B;
    for (int p = 1; p <= h; ++p) {
        for (int idx = threadIdx.x, sx = idx % TW, sy = idx / TW; idx < TW * TH;
             idx += blockDim.x, next_cell(sx, sy, sq, TW)) {
            if (sx < p || sx >= TW - p || sy < p || sy >= TH - p) continue;
            T s = T(0);
            for (int dj = -1; dj <= 1; ++dj) {
                T row = T(0);
                for (int di = -1; di <= 1; ++di) row += (di == 0 ? T(0.5) : T(0.25)) * cur[(sy + dj) * TW + sx + di];
                s += (dj == 0 ? T(0.5) : T(0.25)) * row;
            }
            nxt[idx] = s;
        }
        __syncthreads();
        // outflow ghosts take the new value of their clamped boundary node
        for (int idx = threadIdx.x, sx = idx % TW, sy = idx / TW; idx < TW * TH;
             idx += blockDim.x, next_cell(sx, sy, sq, TW)) {
            if (sx < p || sx >= TW - p || sy < p || sy >= TH - p) continue;
            const int gi = x0 + sx, gj = y0 + sy;
            int cx = sx, cy = sy;
            if (g.bc[0] == ES_BC_OUTFLOW) cx += (gi < 0 ? -gi : (gi >= g.n1 ? g.n1 - 1 - gi : 0));
            if (g.bc[1] == ES_BC_OUTFLOW) cy += (gj < 0 ? -gj : (gj >= g.n2 ? g.n2 - 1 - gj : 0));
            if (cx != sx || cy != sy) nxt[idx] = nxt[cy * TW + cx];
        }
        __syncthreads();
        T* tmp = cur; cur = nxt; nxt = tmp;
    }
    for (int idx = threadIdx.x; idx < FT_X * FT_Y; idx += blockDim.x) {
        const int ix = idx % FT_X, iy = idx / FT_X;
        const int gi = x0 + h + ix, gj = y0 + h + iy;
        if (gi < g.n1 && gj < g.n2) out[gj * g.n1 + gi] = cur[(h + iy) * TW + h + ix];
    }
}

// launchers (the kernel template is instantiated here): 32 x 16 tiles, 256 threads
template <class T>
static void launch_omega_filter_t(const GridParams& g, const MonitorParams& mp, const T* t0, const T* t1,
                                  const T* t2, const DevScalars* d, int passes, T* out, cudaStream_t s) {
    const dim3 tiles((g.n1 + FT_X - 1) / FT_X, (g.n2 + FT_Y - 1) / FT_Y);
    k_omega_filter_t<T><<<tiles, 256, 0, s>>>(g, mp, t0, t1, t2, d, passes, out);
}
void launch_omega_filter(const GridParams& g, const MonitorParams& mp, const float* t0, const float* t1,
                         const float* t2, const DevScalars* d, int passes, float* out, cudaStream_t s) {
    launch_omega_filter_t(g, mp, t0, t1, t2, d, passes, out, s);
}

__global__ void __launch_bounds__(256) k_jacobi_multi_f(GridParams g, const float* omega, const float* d0,
                                                        float* dout, int sweeps, DevScalars* dv, int limit) {
    __shared__ float Wm[FT_W * FT_H];
    __shared__ float X[2][2][FT_W * FT_H];          // [buffer][component]
    const int h = sweeps, TW = FT_X + 2 * h, TH = FT_Y + 2 * h;
    const int2 sq = make_int2(int(blockDim.x) % TW, int(blockDim.x) / TW);
    const int x0 = blockIdx.x * FT_X - h, y0 = blockIdx.y * FT_Y - h;
    for (int idx = threadIdx.x, sx = idx % TW, sy = idx / TW; idx < TW * TH;
         idx += blockDim.x, next_cell(sx, sy, sq, TW)) {
        const int gi = x0 + sx, gj = y0 + sy;
        Wm[idx] = field_at_f(g, omega, gi, gj);
        X[0][0][idx] = disp_at(g, d0, gi, gj, 0);
        X[0][1][idx] = disp_at(g, d0, gi, gj, 1);
    }
    __syncthreads();
    const float ih2x = float(g.inv_dxi[0] * g.inv_dxi[0]), ih2y = float(g.inv_dxi[1] * g.inv_dxi[1]);
    const float dxx = float(1.0 / g.inv_dxi[0]), dxy = float(1.0 / g.inv_dxi[1]);
    int b = 0;
    for (int p = 1; p <= h; ++p) {
        const float* c0 = X[b][0];
        const float* c1 = X[b][1];
        float* n0 = X[b ^ 1][0];
        float* n1 = X[b ^ 1][1];
        for (int idx = threadIdx.x, sx = idx % TW, sy = idx / TW; idx < TW * TH;
             idx += blockDim.x, next_cell(sx, sy, sq, TW)) {
            if (sx < p || sx >= TW - p || sy < p || sy >= TH - p) continue;
            const int gi = x0 + sx, gj = y0 + sy;
            const bool outside = (g.bc[0] == ES_BC_OUTFLOW && (gi < 0 || gi >= g.n1)) ||
                                 (g.bc[1] == ES_BC_OUTFLOW && (gj < 0 || gj >= g.n2));
            if (outside || fixed_node_f(g, gi, gj)) {
                n0[idx] = c0[idx];
                n1[idx] = c1[idx];
                continue;
            }
            const float w0 = Wm[idx];
            float den = 0.0f, num0 = 0.0f, num1 = 0.0f;
            {   // direction 1
                const float wp = 0.5f * (w0 + Wm[idx + 1]) * ih2x;
                const float wm = 0.5f * (w0 + Wm[idx - 1]) * ih2x;
                den += wp + wm;
                num0 += wp * (c0[idx + 1] + dxx) + wm * (c0[idx - 1] - dxx);
                num1 += wp * (c1[idx + 1] + 0.0f) + wm * (c1[idx - 1] - 0.0f);
            }
            {   // direction 2
                const float wp = 0.5f * (w0 + Wm[idx + TW]) * ih2y;
                const float wm = 0.5f * (w0 + Wm[idx - TW]) * ih2y;
                den += wp + wm;
                num0 += wp * (c0[idx + TW] + 0.0f) + wm * (c0[idx - TW] - 0.0f);
                num1 += wp * (c1[idx + TW] + dxy) + wm * (c1[idx - TW] - dxy);
            }
            const float idn = 1.0f / den;
            n0[idx] = num0 * idn;
            n1[idx] = num1 * idn;
        }
        __syncthreads();
        b ^= 1;
    }
    const size_t N = size_t(g.n1) * g.n2;
    float lim = 1.0f;                                        // limit: k_limiter_f's min over this tile's nodes
    for (int idx = threadIdx.x; idx < FT_X * FT_Y; idx += blockDim.x) {
        const int ix = idx % FT_X, iy = idx / FT_X;
        const int gi = x0 + h + ix, gj = y0 + h + iy;
        if (gi < g.n1 && gj < g.n2) {
            const int s = (h + iy) * TW + h + ix;
            const size_t id = size_t(gj) * g.n1 + gi;
            dout[id] = X[b][0][s];
            dout[N + id] = X[b][1][s];
            if (limit) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float d0k = d0[k * N + id];
                    const float dx = X[b][k][s] - d0k;
                    const int di = k == 0, dj = k == 1;
                    const float hk = k == 0 ? dxx : dxy;
                    if (dx < 0.0f) lim = fminf(lim, -(hk + d0k - disp_at(g, d0, gi - di, gj - dj, k)) / (2.0f * dx));
                    else if (dx > 0.0f) lim = fminf(lim, (hk + disp_at(g, d0, gi + di, gj + dj, k) - d0k) / (2.0f * dx));
                }
            }
        }
    }
    if (limit) {
        lim = block_min_f32(lim);
        if (threadIdx.x == 0) atomic_min_pos(&dv->red[RED_GAMMA], double(lim));
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) atomicAdd(&dv->sweeps, sweeps);
}

}  // namespace es
