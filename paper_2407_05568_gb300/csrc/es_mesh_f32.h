// es_mesh_f32.h -- time step and mesh redistribution of the mixed form on the FP32 pipe.
#pragma once
#include <cuda_runtime.h>

#include "es_aux.h"
#include "es_df.cuh"

namespace es {

// float copies of the gas constants, and the (hi, lo) pairs the monitor's G is evaluated with
struct GasF32 {
    float a, b, R, cv, delta, icv;
    mixed::GasDF gdf;
};

inline GasF32 gas_f32(const Gas& g) {
    GasF32 f;
    f.a = float(g.a);
    f.b = float(g.b);
    f.R = float(g.R);
    f.cv = float(g.cv);
    f.delta = float(g.delta);
    f.icv = float(1.0 / g.cv);
    f.gdf = mixed::gas_df(g.a, g.b, g.R, g.cv);
    return f;
}

// JU, J: the mixed form's (hi, lo) float planes; disp: the FP32 displacement [dim][N]
// vel (nullable): the float mesh velocity; slot: RED_CFL (mesh at rest) or RED_CFL2 (with the step's velocity)
__global__ void k_cfl_f(GridParams g, GasF32 G, const float* JU, const float* J, const float* disp, const float* vel,
                        int slot, DevScalars* d);
// rhoF, GF: 2 N floats each, (hi, lo) planes of the density and the fundamental derivative
__global__ void k_mon_fields_f(GridParams g, GasF32 G, const float* JU, const float* J, float* rhoF, float* GF);
// monitor terms over tiles of MON_NT threads (k_mon_f, 32 x 8 or 30 x 6 nodes, chosen by the mesh size)
// do_dt: 0 no time step; 1 the step's dt from the CFL maximum an earlier kernel left (k_dt's work); 2 also eq. cfl
// with the mesh at rest at every node (k_cfl_f's work on disp, its moving-pass terms to cfl_terms when non-null)
// and dt set by the last block to finish; the last block also forms omega's coefficients (DevScalars::mon_c)
constexpr int MON_NT = 256;
void launch_mon_f(const GridParams& g, const GasF32& G, const float* JU, const float* J, const MonitorParams& mp,
                  float* t0, float* t1, float* t2, DevScalars* d, int do_dt, double cfl, double dt_fixed,
                  const float* disp, float* cfl_terms, int nsm, cudaStream_t s);
__global__ void k_mon_omega_f(GridParams g, MonitorParams mp, const float* t0, const float* t1, const float* t2,
                              const DevScalars* d, float* omega);
__global__ void k_filter_f(GridParams g, const float* in, float* out);
__global__ void k_jacobi_f(GridParams g, const float* omega, const float* d0, float* da, float* db, int k,
                           DevScalars* d, int check, double eps);
__global__ void k_limiter_f(GridParams g, const float* d0, const float* da, const float* db, DevScalars* d);
// fused 2D passes on register tiles 64 nodes wide (halo = the pass or sweep count, 1 .. 8)
// omega and its low-pass filter passes in one launch
void launch_omega_filter(const GridParams& g, const MonitorParams& mp, const float* t0, const float* t1,
                         const float* t2, const DevScalars* d, int passes, float* out, cudaStream_t s);
// sweeps Jacobi sweeps without a tolerance from d0 into dout in one launch; limit: also Delta_gamma of the
// result into RED_GAMMA (k_limiter_f's work)
void launch_jacobi_tiles(const GridParams& g, const float* omega, const float* d0, float* dout, int sweeps,
                         DevScalars* dv, int limit, cudaStream_t s);
// cfl > 0: also eq. cfl with the new velocity from k_cfl_f's stored terms into RED_CFL2, and
// dt = min(dt, cfl / that maximum)
__global__ void k_velocity_f(GridParams g, const float* __restrict__ d0, const float* __restrict__ da,
                             const float* __restrict__ db, DevScalars* d, float* __restrict__ fxd,
                             double* __restrict__ xdot, const float* __restrict__ terms, double cfl);

}  // namespace es
