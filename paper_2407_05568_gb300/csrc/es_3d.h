// es_3d.h -- the three-dimensional FP64 path: metrics, node fields, direction-split flux
// kernels and the mesh redistribution on an n1 x n2 x n3 mesh ([comp][n3][n2][n1], xi_1 fastest).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "es_aux.h"
#include "es_device.cuh"

namespace es {

struct Grid3 {
    int n[3];
    int bc[3];
    double inv_dxi[3];
    double period[3];
    float finv[3], finv2[3];    // 1/dxi_k and 1/dxi_k^2 rounded once to float on the host (the FP32 kernels' copies)
};

// the context's 3D scratch (device) and settings
struct Ctx3 {
    Grid3 g;
    Gas gas;
    Weno weno;
    MonitorParams mon;
    int diss;
    int mixed;                // ES_PREC_MIXED: double-float state, FP32 direction kernels (es_3d_mixed.cu)
    int filter_passes, sweeps;
    double eps;
    int grid;                 // blocks of the grid-stride kernels
    int shape;                // pencil shape of the direction kernels (D3_NSHAPES of them, see es_3d.cu)
    size_t N;                 // nodes
    size_t NE;                // nodes of the grid extended by 3 ghosts in every direction
    size_t NKk[3];            // nodes of direction k's metric grid (3 ghosts along xi_k only)
    double* XE;               // stage coordinates on the extended grid [3][NE]
    double* D;                // cross-form products delta_l[x_p] x_q on the extended grid [9][NE] (k3_deriv)
    double* NK[3];            // J dxi_k/dx_j on direction k's metric grid [3][NKk] (mixed form: floats)
    double* NF;               // node fields of the stage state [F3_COUNT][N] (mixed: float fields)
    double* RH;               // right-hand sides accumulated over the directions [6][N] (mixed: float)
    // mesh scratch (the context's buffers)
    double *rhoF, *GF, *t0, *t1, *t2, *om0, *om1, *xa, *xb;
    float* gc;                // mixed form: the sweeps' constant term g [3][N]
    float* XD;                // mixed form: the step's mesh velocity on the extended mesh [3][NE] (float)
    // mixed form: tensor maps (CUtensorMap, 128 bytes) of the float node fields for the TMA-staged xi_2 and
    // xi_3 pencils, per direction and pencil shape; state 0 = not built yet, 1 = built, -1 = plain loads
    int no_tma;               // 1: plain loads only (tile D3_NSHAPES + k)
    unsigned char tmap[2][4][128];
    int tmap_state[2][4];
};

// arguments of one operator evaluation / RK stage
struct Stage3 {
    const void *JUn, *Jn, *JUs, *Js;    // double, or the mixed form's double-float planes
    const double *xn, *xdot;  // mesh at t^n and its velocity (xdot nullable)
    void *JUo, *Jo;
    double ca, cb, cst;       // Shu-Osher coefficients and the stage time fraction
    double dt_host;
    const double* dt_dev;     // device dt (nullptr: dt_host)
    int mode;                 // 0: RK combination; 1: right-hand sides into (JUo, Jo)
    int reuse;                // the metrics and node fields of (xn, JUs, Js) are in the buffers
    // mixed form, within a step: the metric coordinates (d->XE) hold x^n + xe_cst dt xdot, so the stage's are
    // formed by adding (cst - xe_cst) dt xdot (xe_incr); xd_ready: d->XD already holds xdot on the extended mesh
    // (else the stage forms it first: the metrics' increments and the direction kernels read it)
    int xe_incr, xd_ready;
    double xe_cst;
};

constexpr int D3_NSHAPES = 4;
static_assert(D3_NSHAPES == 4, "Ctx3::tmap holds one tensor map per direction and pencil shape");
cudaError_t d3_alloc(Ctx3* d);
void d3_free(Ctx3* d);
cudaError_t d3_prepare();
// each returns the number of kernels it launched (negative: a launch failed, *err set)
int d3_init_J(const Ctx3* d, const double* x, void* J, cudaStream_t s, cudaError_t* err);
int d3_stage(Ctx3* d, const Stage3& a, DevStatus* st, cudaStream_t s, cudaError_t* err);
int d3_cfl(Ctx3* d, const void* JU, const void* J, const double* x, DevScalars* dv, cudaStream_t s,
           cudaError_t* err);
// xe_current: the stage-metric coordinates of xn (d->XE) are current (the step's d3_cfl just formed them)
int d3_mesh(Ctx3* d, const void* JU, const void* J, const double* xn, double* xdot, DevScalars* dv,
            cudaStream_t s, cudaError_t* err, bool xe_current = false);
// eq. cfl with the step's mesh velocity (into RED_CFL2), from the node fields and metrics d3_cfl left for x^n
int d3_cfl_moving(Ctx3* d, const void* J, const double* xdot, DevScalars* dv, cudaStream_t s, cudaError_t* err);
// the mixed form's kernels (es_3d_mixed.cu)
cudaError_t d3f_prepare();
// the stage metrics of the mixed form (double-float arithmetic, float metrics in NK[k] as [3][NKk])
int d3f_metrics(Ctx3* d, const double* xn, const double* xdot, double cst, const double* dt_dev, double dt_host,
                cudaStream_t s, const Stage3* inc = nullptr);
int d3f_nodes(Ctx3* d, const void* JU, const void* J, DevStatus* st, cudaStream_t s);
int d3f_cfl(Ctx3* d, const void* J, const double* xdot, int slot, DevScalars* dv, cudaStream_t s);
int d3f_init_J(Ctx3* d, const double* Jd, void* J, cudaStream_t s);
int d3f_directions(Ctx3* d, const Stage3& a, DevStatus* st, cudaStream_t s, cudaError_t* err);
// xdot on the extended mesh as floats into d->XD (the coordinates' ghost rule without the period shift)
int d3f_form_xd(Ctx3* d, const double* xdot, cudaStream_t s);
int d3f_mesh(Ctx3* d, const void* JU, const void* J, const double* xn, double* xdot, DevScalars* dv,
             cudaStream_t s, cudaError_t* err, bool xe_current);

}  // namespace es
