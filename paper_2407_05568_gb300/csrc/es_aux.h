// es_aux.h -- declarations of the auxiliary kernels (init, time step, mesh).
#pragma once
#include <cuda_runtime.h>

#include "es_device.cuh"

namespace es {

struct GridParams {
    int dim;
    int n1, n2;
    int bc[2];
    double inv_dxi[2];
    double period[2];
    // float copies formed on the host (grid_floats): 1/dxi_k, dxi_k and 1/dxi_k^2, each the double value rounded
    // once; the FP32 kernels read these instead of converting (double conversions and divisions issue at 1/64 of
    // the FP32 rate on this GPU)
    float finv[2], fdx[2], finv2[2];
    double dx[2];       // 1 / inv_dxi_k (host-formed, as the kernels formed it)
    float dxh[2], dxl[2];   // dx_k as the unevaluated float sum dxh + dxl
};

inline void grid_floats(GridParams& g) {
    for (int k = 0; k < 2; ++k) {
        g.finv[k] = float(g.inv_dxi[k]);
        g.fdx[k] = float(1.0 / g.inv_dxi[k]);
        g.finv2[k] = float(g.inv_dxi[k] * g.inv_dxi[k]);
        g.dx[k] = 1.0 / g.inv_dxi[k];
        g.dxh[k] = float(g.dx[k]);
        g.dxl[k] = float(g.dx[k] - double(g.dxh[k]));
    }
}

struct MonitorParams {
    int kind;            // ES_MONITOR_*
    int kappa;
    double w0, w1, w2;   // weights of the three monitor terms
};

// RED_CFL: eq. cfl's maximum with the mesh at rest; RED_CFL2: the same with the step's mesh velocity
enum { RED_CFL = 0, RED_MON0 = 1, RED_MON1 = 2, RED_MON2 = 3, RED_GAMMA = 4, RED_JAC = 5, RED_JAC2 = 6, RED_CFL2 = 7 };

// Device-resident scalars of a run.
struct DevScalars {
    double t, dt, t_end, last_dt, gamma;
    unsigned long long red[8];
    int sweeps;          // Jacobi sweeps of the current solve
    int conv;            // the current solve reached its tolerance
    int pick;            // 1: the warm start was kept
    unsigned int done;   // blocks finished (last-block reductions)
    DevStatus status;
    double last_change[2];                     // first-sweep changes from x_n and from the warm start
    long long sweeps_total, solves, warm_kept; // cumulative mesh-solve counters
    float mon_c[3];      // mixed form: omega's coefficients alpha_k / max_k as floats (k_mon_f's last block)
    double base[2];      // mixed form: the origin (x_00, y_00) the step's FP32 displacement is measured from
};

// the per-step reset of the reductions and counters (k_reset), and the time step from the CFL
// maximum clipped to the end time (k_dt); one thread runs each
__device__ __forceinline__ void reset_scalars(DevScalars* d) {
    for (int k = 0; k < 8; ++k) d->red[k] = 0ULL;
    d->red[RED_GAMMA] = (unsigned long long)__double_as_longlong(1.0);
    d->sweeps = 0;
    d->conv = 0;
    d->pick = 0;
    d->done = 0u;
}

__device__ __forceinline__ void set_dt_from_max(DevScalars* d, double mx, double cfl, double dt_fixed) {
    double dt = dt_fixed > 0.0 ? dt_fixed : cfl / mx;
    const double left = d->t_end - d->t;
    if (left <= 1e-14 * fmax(1.0, fabs(d->t_end))) dt = 0.0;
    else if (dt > left) dt = left;
    d->dt = dt;
}
__device__ __forceinline__ void set_dt_from_cfl(DevScalars* d, double cfl, double dt_fixed) {
    set_dt_from_max(d, __longlong_as_double((long long)d->red[RED_CFL]), cfl, dt_fixed);
}

// eq. cfl with the step's mesh velocity (maximum mx): Delta t_n = min(Delta t^(0), CFL / mx).
// The mesh velocity keeps its value, so the mesh moves Delta_gamma' dx with Delta_gamma' <= Delta_gamma.
__device__ __forceinline__ void shrink_dt_to(DevScalars* d, double mx, double cfl) {
    const double dt = cfl / mx;
    if (d->dt > 0.0 && dt < d->dt) d->dt = dt;
}
__device__ __forceinline__ void shrink_dt_for_mesh(DevScalars* d, double cfl) {
    shrink_dt_to(d, __longlong_as_double((long long)d->red[RED_CFL2]), cfl);
}

// eq. cfl's node term with a mesh velocity from the terms the mesh-at-rest pass stored: per direction k,
// S_k = (n_k . v) f_k, P_k = n_k1 f_k, Q_k = n_k2 f_k, C_k = |n_k| c f_k with f_k = 1/(J dxi_k), fields
// 0..3 (k = 1) in t0 and 4..7 (k = 2) in t1; in 1D S, P, C in t0.  C_k is HUGE at a node without a real
// sound speed.  The term is sum_k |S_k - (xdot_1 P_k + xdot_2 Q_k)| + C_k.
template <class T>
__device__ __forceinline__ T cfl_moving_term(const T* t0, const T* t1, size_t N, size_t id, int dim, T xd1, T xd2) {
    if (dim == 1) return fabs(t0[id] - xd1 * t0[N + id]) + t0[2 * N + id];
    return fabs(t0[id] - (xd1 * t0[N + id] + xd2 * t0[2 * N + id])) + t0[3 * N + id] +
           fabs(t1[id] - (xd1 * t1[N + id] + xd2 * t1[2 * N + id])) + t1[3 * N + id];
}

// kernels templated on the state type are launched through these (f32: float state)
void launch_init_J(const GridParams& g, const double* x, void* J, bool f32, int grid, cudaStream_t s);
void launch_prim_to_cons(const GridParams& g, const Gas& G, const double* rho, const double* v, const double* p,
                         const void* J, void* JU, bool f32, int grid, cudaStream_t s);
// xdot (nullable): the mesh velocity of eq. VCLCoeff's J xi_t; slot: RED_CFL or RED_CFL2; t0, t1 (nullable):
// also store the node terms cfl_moving_term reads (mesh at rest only); rhoF, GF (nullable): also the monitor's
// fields (k_mon_fields' work); set_dt: the last block also sets dt from the maximum (k_dt's work)
void launch_cfl(const GridParams& g, const Gas& G, const void* JU, const void* J, const double* x,
                const double* xdot, int slot, DevScalars* d, bool f32, int grid, cudaStream_t s,
                double* t0 = nullptr, double* t1 = nullptr, int block = 256, double* rhoF = nullptr,
                double* GF = nullptr, int set_dt = 0, double cfl = 0.0, double dt_fixed = 0.0);
// total entropy rate sum_i (V_i . d(JU)_i/dt - phi_i dJ_i/dt) vol in FP64 with a compensated, fixed-order
// reduction: out[0] the rate, out[1] the sum of the magnitudes of its terms (device); part holds 3 grid doubles
void launch_entropy_rate(int N, int dim, const Gas& G, const void* JU, const void* J, const void* dJU,
                         const void* dJ, double vol, double* part, double* out, bool f32, int grid, cudaStream_t s);
void launch_mon_fields(const GridParams& g, const Gas& G, const void* JU, const void* J, double* rhoF, double* GF,
                       bool f32, int grid, cudaStream_t s, int block = 256);
__global__ void k_reset(DevScalars* d);
__global__ void k_dt(DevScalars* d, double cfl, double dt_fixed);
__global__ void k_dt_moving(DevScalars* d, double cfl);
__global__ void k_set_dt(DevScalars* d, double dt);
__global__ void k_set_t_end(DevScalars* d, double t_end);
// x += dt xdot and t += dt; fdisp (nullable): also the FP32 displacement of the new x from d->base (the next
// step's, as k_mesh_f32 forms it); reset: also reset the next step's reductions (k_reset's work)
__global__ void k_advance(GridParams g, double* x, const double* xdot, DevScalars* d, float* fdisp = nullptr,
                          int reset = 0);
// rst (nullable): also runs k_reset's work (the first kernel of a mixed-form step)
// fxd is written only when xdot is given (its readers take it only then)
__global__ void k_mesh_f32(GridParams g, const double* __restrict__ x, const double* __restrict__ xdot,
                           float* __restrict__ disp, float* __restrict__ fxd, DevScalars* rst = nullptr);
__global__ void k_mon_terms(GridParams g, MonitorParams mp, const double* rhoF, const double* GF, double* t0,
                            double* t1, double* t2, DevScalars* d);
__global__ void k_mon_omega(GridParams g, MonitorParams mp, const double* t0, const double* t1, const double* t2,
                            const DevScalars* d, double* omega);
__global__ void k_filter(GridParams g, const double* in, double* out);
__global__ void k_jacobi(GridParams g, const double* omega, const double* first, double* xa, double* xb, int k,
                         int dst0, DevScalars* d, int check, int slot, int decide, double eps, int limit = 0);
__global__ void k_jacobi_loop(GridParams g, const double* omega, const double* xn, double* xa, double* xb,
                              DevScalars* d, double eps, int mu, cudaGraphConditionalHandle h);
__global__ void k_pick(DevScalars* d, int check, double eps, double ratio);
__global__ void k_limiter(GridParams g, const double* xn, const double* xa, const double* xb, DevScalars* d);
// cfl > 0: also eq. cfl with the new velocity from the stored terms (t0, t1) into RED_CFL2, and the last block
// shrinks dt to it
__global__ void k_velocity(GridParams g, const double* xn, const double* xa, const double* xb, DevScalars* d,
                           double* xdot, const double* t0 = nullptr, const double* t1 = nullptr, double cfl = 0.0);
__global__ void k_jacobi_out(GridParams g, const double* xn, const double* xa, const double* xb,
                             const DevScalars* d, double* xout, float* disp);
__global__ void k_features(GridParams g, const double* omega, const double* GF, const double* x, float* feat);
__global__ void k_warm_start(GridParams g, const double* xn, const float* out, double* x0);

}  // namespace es
