// es_api.cu -- the C ABI (include/es_vdw.h): context, argument checks, step
// sequencing, CUDA-graph replay and error reporting.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "es_3d.h"
#include "es_aux.h"
#include "es_internal.h"
#include "es_mesh_f32.h"
#include "es_vdw.h"

using namespace es;

struct es_ctx {
    es_params p;
    int device;
    cudaStream_t stream;              // the caller's stream
    cudaStream_t s_enq;               // stream the enqueue helpers launch on (capture stream while capturing)
    cudaStream_t cap_stream;          // private stream for graph capture (the legacy stream cannot capture)
    cudaStream_t body_stream;         // captures the body of a graph while-loop
    GridParams g;
    Gas gas;
    Weno weno;
    MonitorParams mon;
    size_t N;
    int nc;
    int grid1d;                       // blocks of the per-node grid-stride kernels
    int block1d;                      // their threads per block (see es_create)
    int nsm;                          // SMs of the device
    double t_end_dev;                 // the end time the device holds (NaN: unknown)
    int mixed;                        // ES_PREC_MIXED: float state
    int tile;                         // 2D stage tile shape (0-based); tuned: chosen by es_autotune or fixed
    int tuned;
    size_t esz;                       // bytes per state element (8 or 4)
    // scratch (device)
    void *S1, *S1J, *S2, *S2J;        // RK stage states in the state precision
    float *fdisp, *fxd;               // mixed form: FP32 mesh displacement and velocity
    double *rhoF, *GF, *t0, *t1, *t2, *om0, *om1;
    double *xa, *xb, *xdot;
    // learned warm start (2D): network copy (float weights), features, activations
    int nn_layers, nn_hidden;
    double nn_ratio;                  // guard: keep the warm start if c1 < nn_ratio c0
    uint16_t* nn_wbf;                 // bf16 weights (the context's copy)
    float *nn_b, *feat, *act0, *act1, *nn_out;
    double* xw;
    DevScalars* dev;
    DevScalars* hpin;                 // pinned host mirror
    void *hJU, *hJ;                   // device copies for es_run_host
    double* hx;
    // graph cache
    // the step graphs: [0] a call's only step, [1] the first of several (its advance kernel also forms the next
    // step's displacement and resets the reductions), [2] the steps after it (1D/2D: without the displacement or
    // reset kernel at their start)
    cudaGraphExec_t gexec[3];
    const void* gkey[3];
    int graph_kernels[3];
    int capturing;
    int capture_count;
    int loop_failed;                  // a graph while-loop could not be built (unrolled sweeps used)
    int64_t launches;
    Ctx3* d3;                         // the 3D path's scratch and settings (dim = 3)
    char msg[256];
};

// the cached step graphs (they hold the buffers, the tile shape and the warm-start network)
static void drop_graphs(es_ctx* c) {
    for (int k = 0; k < 3; ++k) {
        if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
        c->gexec[k] = nullptr;
    }
}


namespace {

int fail(es_ctx* c, int code, const char* what) {
    if (c) snprintf(c->msg, sizeof(c->msg), "%s", what);
    return code;
}

int cuda_fail(es_ctx* c, cudaError_t e, const char* where) {
    if (c) snprintf(c->msg, sizeof(c->msg), "%s: %s", where, cudaGetErrorString(e));
    return ES_ERR_CUDA;
}

#define CK(call, where)                              \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

void count(es_ctx* c, int n = 1) {
    if (c->capturing) c->capture_count += n;
    else c->launches += n;
}

StageParams stage_params(es_ctx* c) {
    StageParams P;
    memset(&P, 0, sizeof(P));
    P.dim = c->p.dim;
    P.n1 = c->p.n1;
    P.n2 = c->p.n2;
    P.bc[0] = c->p.bc[0];
    P.bc[1] = c->p.bc[1];
    P.inv_dxi[0] = 1.0 / c->p.dxi[0];
    P.inv_dxi[1] = c->p.dim == 2 ? 1.0 / c->p.dxi[1] : 0.0;
    P.period[0] = c->p.period[0];
    P.period[1] = c->p.period[1];
    P.gas = c->gas;
    P.weno = c->weno;
    P.diss = c->p.dissipation;
    P.status = &c->dev->status;
    P.tile = c->tile;
    return P;
}

// state pointers of a stage launch in the context's precision
void set_state(es_ctx* c, StageParams& P, const void* JUn, const void* Jn, const void* JUs, const void* Js,
               void* JUo, void* Jo) {
    if (c->mixed) {
        P.fJUn = (const float*)JUn;
        P.fJn = (const float*)Jn;
        P.fJUs = (const float*)JUs;
        P.fJs = (const float*)Js;
        P.fJUo = (float*)JUo;
        P.fJo = (float*)Jo;
    } else {
        P.JUn = (const double*)JUn;
        P.Jn = (const double*)Jn;
        P.JUs = (const double*)JUs;
        P.Js = (const double*)Js;
        P.JUo = (double*)JUo;
        P.Jo = (double*)Jo;
    }
}

// mixed form: FP32 mesh displacement / velocity for the stage kernels
void enqueue_mesh_f32(es_ctx* c, StageParams& P, const double* x, const double* xdot) {
    if (!c->mixed) return;
    k_mesh_f32<<<c->grid1d, c->block1d, 0, c->s_enq>>>(c->g, x, xdot, c->fdisp, c->fxd);
    count(c);
    P.fdisp = c->fdisp;
    P.fxdot = xdot ? c->fxd : nullptr;
}

cudaError_t launch_stage(es_ctx* c, const StageParams& P) {
    count(c);
    if (c->mixed) {
        StageParams Q = P;
        set_float_params(Q);
        return launch_stage_mixed(Q, c->s_enq);
    }
    return launch_stage_fp64(P, c->s_enq);
}

const double RK_A[3] = {0.0, 0.75, 1.0 / 3.0};
const double RK_B[3] = {1.0, 0.25, 2.0 / 3.0};
const double RK_C[3] = {0.0, 1.0, 0.5};

// monitor -> filter passes (Sec. 4); returns the buffer holding the filtered omega
// fields_ready: the step's CFL kernel already wrote rho and G (c->rhoF, c->GF) for this state
const double* enqueue_monitor(es_ctx* c, const void* JU, const void* J, bool fields_ready = false) {
    const int B = c->block1d, G = c->grid1d;
    cudaStream_t s = c->s_enq;
    if (!fields_ready) {
        launch_mon_fields(c->g, c->gas, JU, J, c->rhoF, c->GF, c->mixed, G, s, B);
        count(c);
    }
    k_mon_terms<<<G, B, 0, s>>>(c->g, c->mon, c->rhoF, c->GF, c->t0, c->t1, c->t2, c->dev);
    k_mon_omega<<<G, B, 0, s>>>(c->g, c->mon, c->t0, c->t1, c->t2, c->dev, c->om0);
    count(c, 2);
    double* om = c->om0;
    double* other = c->om1;
    for (int k = 0; k < c->p.filter_passes; ++k) {
        k_filter<<<G, B, 0, s>>>(c->g, om, other);
        count(c);
        double* tmp = om; om = other; other = tmp;
    }
    return om;
}

// learned warm start x0 = x_n + dxi NN(features) into c->xw
int enqueue_net(es_ctx* c, const double* om, const double* xn) {
    const int B = c->block1d, G = c->grid1d;
    cudaStream_t s = c->s_enq;
    k_features<<<G, B, 0, s>>>(c->g, om, c->GF, xn, c->feat);
    count(c);
    const float* in = c->feat;
    int cin = c->p.dim + 2;
    size_t woff = 0, boff = 0;
    for (int l = 0; l < c->nn_layers; ++l) {
        const bool last = l == c->nn_layers - 1;
        const int cout = last ? c->p.dim : c->nn_hidden;
        float* out = last ? c->nn_out : ((l & 1) ? c->act1 : c->act0);
        // layer inputs after the first and outputs before the last stay bf16 [H][W][C]
        cudaError_t e = nn_conv_forward_bf16_fmt(in, l > 0, c->nn_wbf + woff, c->nn_b + boff, out, !last, 1, cin,
                                                 cout, c->g.n2, c->g.n1, last ? 0 : 1, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "warm-start network");
        count(c);
        woff += size_t(cout) * cin * 9;
        boff += cout;
        in = out;
        cin = cout;
    }
    k_warm_start<<<G, B, 0, s>>>(c->g, xn, c->nn_out, c->xw);
    count(c);
    return ES_OK;
}

// While-loop node in the step graph being captured on c->s_enq; its body (one k_jacobi_loop
// launch) is captured on c->body_stream.  Each pass of the loop runs one sweep; the kernel sets
// the loop condition (to 0 once converged or after mu sweeps, so the loop always ends).
// Returns LOOP_OK, LOOP_UNTOUCHED (nothing added: the caller may unroll the sweeps instead) or
// LOOP_BROKEN (a node was added but its body could not be built: the capture must be abandoned,
// since a while-node without the kernel that clears its condition would never end).
enum { LOOP_OK = 0, LOOP_UNTOUCHED = 1, LOOP_BROKEN = 2 };
int enqueue_sweep_loop(es_ctx* c, const double* om, const double* xn) {
    cudaStreamCaptureStatus st;
    cudaGraph_t graph;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(c->s_enq, &st, nullptr, &graph, &deps, &edges, &ndeps) != cudaSuccess ||
        st != cudaStreamCaptureStatusActive)
        return LOOP_UNTOUCHED;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return LOOP_UNTOUCHED;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, graph, deps, edges, ndeps, &cp) != cudaSuccess) return LOOP_UNTOUCHED;
    if (cudaStreamUpdateCaptureDependencies(c->s_enq, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
        cudaSuccess)
        return LOOP_BROKEN;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(c->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        return LOOP_BROKEN;
    k_jacobi_loop<<<c->grid1d, c->block1d, 0, c->body_stream>>>(c->g, om, xn, c->xa, c->xb, c->dev, c->p.jacobi_eps,
                                                         c->p.jacobi_sweeps, h);
    const cudaError_t el = cudaGetLastError();
    count(c);
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->body_stream, &out);
    size_t nodes = 0;
    if (el != cudaSuccess || e != cudaSuccess || cudaGraphGetNodes(body, nullptr, &nodes) != cudaSuccess ||
        nodes != 1)
        return LOOP_BROKEN;
    return LOOP_OK;
}

// Jacobi sweeps from x_n, or guarded from x_start (the first sweep runs from both starts
// and the start whose sweep changes the mesh less is continued)
// *limited (nullable): set when the last sweep also formed Delta_gamma (sweeps without a tolerance)
int enqueue_jacobi(es_ctx* c, const double* om, const double* xn, const double* x_start, double ratio,
                   bool* limited = nullptr) {
    const int B = c->block1d, G = c->grid1d;
    cudaStream_t s = c->s_enq;
    const int check = c->p.jacobi_eps > 0.0;
    const double eps = c->p.jacobi_eps;
    int k0 = 0;
    if (x_start && c->p.jacobi_sweeps > 0) {
        k_jacobi<<<G, B, 0, s>>>(c->g, om, xn, c->xa, c->xb, 0, 0, c->dev, 1, RED_JAC, 0, eps);
        k_jacobi<<<G, B, 0, s>>>(c->g, om, x_start, c->xa, c->xb, 0, 1, c->dev, 1, RED_JAC2, 0, eps);
        k_pick<<<1, 32, 0, s>>>(c->dev, check, eps, ratio);
        count(c, 3);
        k0 = 1;
    }
    if (check && c->capturing && c->p.jacobi_sweeps > k0) {
        // the remaining sweeps as a while-loop node: no launches after convergence
        const int r = enqueue_sweep_loop(c, om, xn);
        if (r == LOOP_OK) return ES_OK;
        if (r == LOOP_BROKEN) return fail(c, ES_ERR_CUDA, "graph while-loop of the Jacobi sweeps");
        c->loop_failed = 1;
    }
    for (int k = k0; k < c->p.jacobi_sweeps; ++k) {
        const int lim = limited && !check && k == c->p.jacobi_sweeps - 1;
        k_jacobi<<<G, B, 0, s>>>(c->g, om, xn, c->xa, c->xb, k, 0, c->dev, check, RED_JAC, 1, eps, lim);
        count(c);
        if (lim) *limited = true;
    }
    return ES_OK;
}

// monitor -> filter -> [warm start] -> Jacobi -> limiter -> xdot, with dt already in c->dev->dt; cfl_moving > 0:
// the velocity kernel also takes eq. cfl with the new velocity (from the terms the step's first CFL pass left in
// c->S1 and c->S2) and shrinks dt
int enqueue_mesh(es_ctx* c, const void* JU, const void* J, const double* xn, double* xdot, double cfl_moving = 0.0,
                 bool fields_ready = false) {
    const int B = c->block1d, G = c->grid1d;
    cudaStream_t s = c->s_enq;
    const double* om = enqueue_monitor(c, JU, J, fields_ready);
    const double* x_start = nullptr;
    if (c->nn_layers > 0) {
        int rc = enqueue_net(c, om, xn);
        if (rc) return rc;
        x_start = c->xw;
    }
    bool limited = false;
    int rc = enqueue_jacobi(c, om, xn, x_start, c->nn_ratio, &limited);
    if (rc) return rc;
    if (!limited) {
        k_limiter<<<G, B, 0, s>>>(c->g, xn, c->xa, c->xb, c->dev);
        count(c);
    }
    k_velocity<<<G, B, 0, s>>>(c->g, xn, c->xa, c->xb, c->dev, xdot, (const double*)c->S1, (const double*)c->S2,
                               cfl_moving);
    count(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "mesh kernels");
    return ES_OK;
}

// The mixed form runs the time step and the mesh redistribution on the FP32 displacement
// (es_mesh_f32.cu) unless a warm-start network is registered (its features and guarded
// sweeps are the FP64 kernels).
bool mesh_on_fp32(const es_ctx* c) { return c->mixed && c->nn_layers == 0; }

// Sec. 4 on the FP32 pipe; c->fdisp must hold the displacement of x^n.  Writes c->fxd and xdot.
// with_dt: 1, the monitor kernel also sets the step's dt from the CFL maximum (k_dt's work); 2, it also takes
// eq. cfl with the mesh at rest itself (k_cfl_f's work) and stores the moving pass's terms in c->S1.
// cfl_moving > 0: the velocity kernel also takes eq. cfl with the new mesh velocity (from the terms the step's
// first CFL pass left in c->S1) and shrinks dt.  In 2D the sweeps' tile kernel also forms Delta_gamma.
int enqueue_mesh32(es_ctx* c, const void* JU, const void* J, double* xdot, int with_dt, double cfl_moving = 0.0) {
    const int B = c->block1d, G = c->grid1d;
    cudaStream_t s = c->s_enq;
    const GasF32 gf = gas_f32(c->gas);
    float* t0 = (float*)c->t0;
    float* t1 = (float*)c->t1;
    float* t2 = (float*)c->t2;
    float* om = (float*)c->om0;
    float* other = (float*)c->om1;
    float* da = (float*)c->xa;
    float* db = (float*)c->xb;
    launch_mon_f(c->g, gf, (const float*)JU, (const float*)J, c->mon, t0, t1, t2, c->dev, with_dt, c->p.cfl,
                 c->p.dt_fixed, c->fdisp, cfl_moving > 0.0 ? (float*)c->S1 : nullptr, c->nsm, s);
    count(c);
    // 2D: omega with its filter passes, and the sweeps without a tolerance, fused per tile
    const bool fuse = c->p.dim == 2;
    if (fuse && c->p.filter_passes >= 1 && c->p.filter_passes <= 8) {
        launch_omega_filter(c->g, c->mon, t0, t1, t2, c->dev, c->p.filter_passes, om, s);
        count(c);
    } else {
        k_mon_omega_f<<<G, B, 0, s>>>(c->g, c->mon, t0, t1, t2, c->dev, om);
        count(c);
        for (int k = 0; k < c->p.filter_passes; ++k) {
            k_filter_f<<<G, B, 0, s>>>(c->g, om, other);
            count(c);
            float* tmp = om; om = other; other = tmp;
        }
    }
    const int check = c->p.jacobi_eps > 0.0;
    const int mu = c->p.jacobi_sweeps;
    if (fuse && !check && mu >= 1 && mu <= 8) {              // the tile kernel also forms Delta_gamma
        launch_jacobi_tiles(c->g, om, c->fdisp, ((mu - 1) & 1) ? db : da, mu, c->dev, 1, s);
        count(c);
    } else {
        for (int k = 0; k < mu; ++k) {
            k_jacobi_f<<<G, B, 0, s>>>(c->g, om, c->fdisp, da, db, k, c->dev, check, c->p.jacobi_eps);
            count(c);
        }
        k_limiter_f<<<G, B, 0, s>>>(c->g, c->fdisp, da, db, c->dev);
        count(c);
    }
    k_velocity_f<<<G, B, 0, s>>>(c->g, c->fdisp, da, db, c->dev, c->fxd, xdot, (const float*)c->S1, cfl_moving);
    count(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "mesh kernels (FP32)");
    return ES_OK;
}

// fields: also write the monitor's rho and G fields; set_dt: the kernel also sets the step's dt
void enqueue_cfl(es_ctx* c, const void* JU, const void* J, const double* x, const double* xdot = nullptr,
                 int slot = RED_CFL, double* t0 = nullptr, double* t1 = nullptr, bool fields = false,
                 bool set_dt = false) {
    launch_cfl(c->g, c->gas, JU, J, x, xdot, slot, c->dev, c->mixed, c->grid1d, c->s_enq, t0, t1, c->block1d,
               fields ? c->rhoF : nullptr, fields ? c->GF : nullptr, set_dt ? 1 : 0, c->p.cfl, c->p.dt_fixed);
    count(c);
}

// one 3D step: CFL (its metrics and node fields serve stage 1), mesh, three stages, advance
int enqueue_step3(es_ctx* c, double* JU, double* J, double* x) {
    cudaStream_t s = c->s_enq;
    cudaError_t e;
    k_reset<<<1, 32, 0, s>>>(c->dev);
    count(c);
    int n = d3_cfl(c->d3, JU, J, x, c->dev, s, &e);
    if (n < 0) return cuda_fail(c, e, "3D time-step kernels");
    count(c, n);
    k_dt<<<1, 32, 0, s>>>(c->dev, c->p.cfl, c->p.dt_fixed);
    count(c);
    const double* xdot = nullptr;
    if (c->p.moving) {
        n = d3_mesh(c->d3, JU, J, x, c->xdot, c->dev, s, &e, true);     // d3_cfl formed x^n's metric coordinates
        if (n < 0) return cuda_fail(c, e, "3D mesh kernels");
        count(c, n);
        xdot = c->xdot;
        if (!(c->p.dt_fixed > 0.0)) {          // eq. cfl with the step's mesh velocity
            n = d3_cfl_moving(c->d3, J, xdot, c->dev, s, &e);
            if (n < 0) return cuda_fail(c, e, "3D time-step kernels");
            k_dt_moving<<<1, 32, 0, s>>>(c->dev, c->p.cfl);
            count(c, n + 1);
        }
    }
    double* S1 = (double*)c->S1;
    double* S2 = (double*)c->S2;
    double* S1J = (double*)c->S1J;
    double* S2J = (double*)c->S2J;
    const double* srcU[3] = {JU, S1, S2};
    const double* srcJ[3] = {J, S1J, S2J};
    double* dstU[3] = {S1, S2, JU};
    double* dstJ[3] = {S1J, S2J, J};
    for (int st = 0; st < 3; ++st) {
        Stage3 a;
        a.JUn = JU;
        a.Jn = J;
        a.JUs = srcU[st];
        a.Js = srcJ[st];
        a.xn = x;
        a.xdot = xdot;
        a.JUo = dstU[st];
        a.Jo = dstJ[st];
        a.ca = RK_A[st];
        a.cb = RK_B[st];
        a.cst = RK_C[st];
        a.dt_host = 0.0;
        a.dt_dev = &c->dev->dt;
        a.mode = 0;
        a.reuse = st == 0;                 // x_s = x^n and (JU, J)_s = (JU, J)^n: the CFL's buffers
        // mixed form: the metric coordinates hold x^n after the CFL pass and x^n + dt xdot after stage 2, so
        // stages 2 and 3 move them by (c_s - c_{s-1}) dt xdot
        a.xe_incr = st > 0;
        a.xd_ready = st > 0;               // stage 1 forms xdot on the extended mesh (mixed form)
        a.xe_cst = st > 0 ? RK_C[st - 1] : 0.0;
        n = d3_stage(c->d3, a, &c->dev->status, s, &e);
        if (n < 0) return cuda_fail(c, e, "3D stage kernels");
        count(c, n);
    }
    k_advance<<<c->grid1d, c->block1d, 0, s>>>(c->g, x, xdot, c->dev);
    count(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "advance kernel");
    return ES_OK;
}

// first = false: a step that follows one of the same es_steps call, whose advance kernel has already formed the
// mixed form's FP32 displacement of x and reset the reductions (no k_mesh_f32 or k_reset then; 1D/2D); chain: a
// step of the same call follows, so this step's advance kernel does that work
int enqueue_step(es_ctx* c, void* JU, void* J, double* x, bool first = true, bool chain = false) {
    if (c->p.dim == 3) return enqueue_step3(c, (double*)JU, (double*)J, x);
    const int B = c->block1d, G = c->grid1d;
    cudaStream_t s = c->s_enq;
    const bool f32 = mesh_on_fp32(c);
    // eq. cfl with the step's mesh velocity: the first pass (mesh at rest) leaves its node terms in the stage
    // buffers S1 (and S2), free until the first stage, and the velocity kernel takes the second pass from them
    const double cfl_moving = c->p.moving && !(c->p.dt_fixed > 0.0) ? c->p.cfl : 0.0;
    if (f32) {      // the displacement kernel also resets the step's reductions (k_reset's work)
        if (first) {
            k_mesh_f32<<<G, B, 0, s>>>(c->g, x, nullptr, c->fdisp, c->fxd, c->dev);
            count(c);
        }
        if (!c->p.moving) {         // on a moving mesh the monitor kernel takes eq. cfl (with_dt = 2 below)
            k_cfl_f<<<G, B, 0, s>>>(c->g, gas_f32(c->gas), (const float*)JU, (const float*)J, c->fdisp, nullptr,
                                    RED_CFL, c->dev);
            count(c);
        }
    } else {
        if (first) {
            k_reset<<<1, 32, 0, s>>>(c->dev);
            count(c);
        }
        // the CFL kernel also writes the monitor's fields of this state and sets dt (k_mon_fields', k_dt's work)
        enqueue_cfl(c, JU, J, x, nullptr, RED_CFL, cfl_moving > 0.0 ? (double*)c->S1 : nullptr, (double*)c->S2,
                    c->p.moving, true);
    }
    if (f32 && !c->p.moving) {      // on a moving mesh the FP32 monitor kernel sets dt, and k_cfl does in FP64
        k_dt<<<1, 32, 0, s>>>(c->dev, c->p.cfl, c->p.dt_fixed);
        count(c);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "time-step kernels");
    const double* xdot = nullptr;
    if (c->p.moving) {
        int rc = f32 ? enqueue_mesh32(c, JU, J, c->xdot, 2, cfl_moving)
                     : enqueue_mesh(c, JU, J, x, c->xdot, cfl_moving, true);
        if (rc) return rc;
        xdot = c->xdot;
    }
    StageParams P = stage_params(c);
    P.dt_dev = &c->dev->dt;
    P.xn = x;
    P.xdot = xdot;
    if (f32) {
        P.fdisp = c->fdisp;
        P.fxdot = xdot ? c->fxd : nullptr;
    } else {
        enqueue_mesh_f32(c, P, x, xdot);
    }
    const void* srcU[3] = {JU, c->S1, c->S2};
    const void* srcJ[3] = {J, c->S1J, c->S2J};
    void* dstU[3] = {c->S1, c->S2, JU};
    void* dstJ[3] = {c->S1J, c->S2J, J};
    for (int st = 0; st < 3; ++st) {
        P.ca = RK_A[st];
        P.cb = RK_B[st];
        P.cst = RK_C[st];
        set_state(c, P, JU, J, srcU[st], srcJ[st], dstU[st], dstJ[st]);
        e = launch_stage(c, P);
        if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel");
    }
    // the next step's displacement (mixed form) and reductions, for a following step of the same call
    k_advance<<<G, B, 0, s>>>(c->g, x, xdot ? c->xdot : nullptr, c->dev, chain && f32 ? c->fdisp : nullptr, chain);
    count(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "advance kernel");
    return ES_OK;
}

int check_params(const es_params* p) {
    if (!p) return 0;
    if (p->dim < 1 || p->dim > 3) return 0;
    if (p->n1 < 8) return 0;
    if (p->dim == 1 && p->n2 != 1) return 0;
    if (p->dim >= 2 && p->n2 < 8) return 0;
    if (p->dim < 3 && p->n3 != 0 && p->n3 != 1) return 0;
    if (p->dim == 3 && (p->n3 < 8 || p->tile > (p->precision == ES_PREC_MIXED ? 2 * D3_NSHAPES : D3_NSHAPES)))
        return 0;
    const long long n3 = p->dim == 3 ? p->n3 : 1;
    if ((long long)p->n1 * p->n2 * n3 > (1LL << 30)) return 0;
    for (int k = 0; k < p->dim; ++k) {
        if (!(p->dxi[k] > 0.0)) return 0;
        const bool mirror = p->bc[k] == ES_BC_REFLECT || p->bc[k] == ES_BC_SYMMETRY_LO;
        if (p->bc[k] != ES_BC_PERIODIC && p->bc[k] != ES_BC_OUTFLOW && !(mirror && p->precision == ES_PREC_FP64))
            return 0;
        if (p->bc[k] == ES_BC_PERIODIC && !(p->period[k] > 0.0)) return 0;
    }
    if (!(p->R > 0.0) || !(p->cv > 0.0) || !(p->a >= 0.0) || !(p->b >= 0.0)) return 0;
    if (!(p->weno_gamma[0] > 0.0) || !(p->weno_gamma[1] > 0.0) || !(p->weno_gamma[2] > 0.0)) return 0;
    if (!(p->weno_eps > 0.0)) return 0;
    if (!(p->sign_tol >= 0.0) || p->sign_tol > 1e-2) return 0;
    if (!(p->cfl > 0.0) && !(p->dt_fixed > 0.0)) return 0;
    if (p->precision != ES_PREC_FP64 && p->precision != ES_PREC_MIXED) return 0;
    if (p->tile < 0 || (p->dim < 3 && p->tile > ES_NTILES)) return 0;
    if (p->precision == ES_PREC_MIXED && p->dim < 3) {
        // the FP32 displacement (1D/2D) is periodic only when the period is n dxi
        const int nn[2] = {p->n1, p->n2};
        for (int k = 0; k < p->dim; ++k)
            if (p->bc[k] == ES_BC_PERIODIC && fabs(p->period[k] - nn[k] * p->dxi[k]) > 1e-9 * p->period[k]) return 0;
    }
    if (p->moving) {
        if (p->monitor != ES_MONITOR_VDW && p->monitor != ES_MONITOR_SMOOTH) return 0;
        if (p->monitor == ES_MONITOR_VDW && (p->kappa < 1 || p->kappa > 2)) return 0;
        if (p->filter_passes < 0 || p->jacobi_sweeps < 0 || p->jacobi_sweeps > 100000) return 0;
    }
    return 1;
}

}  // namespace

extern "C" {

int es_create(es_ctx** out, const es_params* p, void* stream) {
    if (!out) return ES_ERR_ARG;
    *out = nullptr;
    if (!check_params(p)) return ES_ERR_ARG;
    es_ctx* c = (es_ctx*)calloc(1, sizeof(es_ctx));
    if (!c) return ES_ERR_ARG;
    c->p = *p;
    c->stream = (cudaStream_t)stream;
    c->s_enq = c->stream;
    CK(cudaGetDevice(&c->device), "cudaGetDevice");
    c->g.dim = p->dim;
    c->g.n1 = p->n1;
    c->g.n2 = p->dim == 2 ? p->n2 : 1;
    c->g.bc[0] = p->bc[0];
    c->g.bc[1] = p->dim == 2 ? p->bc[1] : ES_BC_PERIODIC;
    c->g.inv_dxi[0] = 1.0 / p->dxi[0];
    c->g.inv_dxi[1] = p->dim == 2 ? 1.0 / p->dxi[1] : 0.0;
    grid_floats(c->g);
    c->g.period[0] = p->period[0];
    c->g.period[1] = p->period[1];
    c->gas.a = p->a;
    c->gas.b = p->b;
    c->gas.R = p->R;
    c->gas.cv = p->cv;
    c->gas.delta = p->R / p->cv;
    gas_reciprocals(c->gas);
    const double g1 = p->weno_gamma[0], g2 = p->weno_gamma[1], g3 = p->weno_gamma[2];
    const double gs = g1 + g2 + g3;
    c->weno.g1 = g1 / gs;
    c->weno.g2 = g2 / gs;
    c->weno.g3 = g3 / gs;
    c->weno.g12 = g1 / (g1 + g2);
    c->weno.ig22 = (g1 + g2) / g2;
    c->weno.ig3 = gs / g3;
    c->weno.eps = p->weno_eps;
    c->weno.sign_tol = p->sign_tol;
    c->mon.kind = p->monitor;
    c->mon.kappa = p->kappa;
    if (p->monitor == ES_MONITOR_SMOOTH) {
        c->mon.w0 = p->alpha[0];
        c->mon.w1 = 0.0;
        c->mon.w2 = p->alpha[1];
    } else {
        c->mon.w0 = p->alpha[0];
        c->mon.w1 = p->kappa >= 2 ? p->alpha[1] : 0.0;
        c->mon.w2 = p->alpha[p->kappa];
    }
    if (p->dim == 3) {
        // the 1D/2D elementwise kernels see the 3D mesh as N nodes in a row
        c->g.n1 = p->n1 * p->n2 * p->n3;
        c->g.n2 = 1;
        c->g.bc[0] = c->g.bc[1] = ES_BC_PERIODIC;
        c->g.inv_dxi[0] = c->g.inv_dxi[1] = 1.0;
        grid_floats(c->g);
    }
    c->N = size_t(c->g.n1) * c->g.n2;
    c->nc = p->dim + 2;
    c->mixed = p->precision == ES_PREC_MIXED;
    c->tile = p->tile > 0 ? p->tile - 1 : 0;
    c->tuned = p->tile > 0 || p->dim == 1;
    c->esz = c->mixed ? 2 * sizeof(float) : sizeof(double);   // mixed: (hi, lo) float planes
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    c->nsm = nsm;
    c->t_end_dev = __builtin_nan("");
    // The per-node kernels of a step (CFL, monitor, filter, sweeps, limiter, velocity, advance) take one node per
    // thread on a small mesh, so their time is one thread's chain of dependent operations: there every CTA gets its
    // own SM (blocks of ceil(N / SMs) threads, at most 512; with 256-thread blocks 200^2 gave 157 CTAs on 152 SMs
    // and a few SMs ran two, doubling the launch).  Larger meshes take 256-thread blocks, at most 8 per SM.
    const size_t per_sm = (c->N + size_t(nsm) - 1) / size_t(nsm);
    if (per_sm <= 512) {
        c->block1d = int((per_sm + 31) / 32 * 32);
        if (c->block1d < 64) c->block1d = 64;
        c->grid1d = int((c->N + size_t(c->block1d) - 1) / size_t(c->block1d));
    } else {
        const size_t blocks = (c->N + 255) / 256;
        c->block1d = 256;
        c->grid1d = (int)(blocks < size_t(nsm) * 8 ? blocks : size_t(nsm) * 8);
    }
    if (c->grid1d < 1) c->grid1d = 1;
    const size_t B = sizeof(double) * c->N;
    int rc = ES_OK;
#define ALLOC(ptr, bytes)                                                            \
    do {                                                                             \
        cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                         \
        if (e_ != cudaSuccess) { rc = cuda_fail(c, e_, "cudaMalloc"); goto fail_out; } \
    } while (0)
    ALLOC(c->S1, c->esz * c->N * c->nc);
    ALLOC(c->S2, c->esz * c->N * c->nc);
    ALLOC(c->S1J, c->esz * c->N);
    ALLOC(c->S2J, c->esz * c->N);
    if (c->mixed) {
        ALLOC(c->fdisp, sizeof(float) * c->N * p->dim);
        ALLOC(c->fxd, sizeof(float) * c->N * p->dim);
    }
    ALLOC(c->rhoF, B);
    ALLOC(c->GF, B);
    ALLOC(c->t0, B);
    ALLOC(c->t1, B);
    ALLOC(c->t2, B);
    ALLOC(c->om0, B);
    ALLOC(c->om1, B);
    ALLOC(c->xa, B * p->dim);
    ALLOC(c->xb, B * p->dim);
    ALLOC(c->xdot, B * p->dim);
    ALLOC(c->dev, sizeof(DevScalars));
#undef ALLOC
    {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->body_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { rc = cuda_fail(c, e, "cudaStreamCreate"); goto fail_out; }
        e = cudaMallocHost((void**)&c->hpin, sizeof(DevScalars));
        if (e != cudaSuccess) { rc = cuda_fail(c, e, "cudaMallocHost"); goto fail_out; }
        e = cudaMemsetAsync(c->dev, 0, sizeof(DevScalars), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->xdot, 0, B * p->dim, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { rc = cuda_fail(c, e, "init"); goto fail_out; }
        // warm the stage kernel once so its shared-memory attribute is set outside any capture
        if (p->dim == 3) {
            e = d3_prepare();
            if (e == cudaSuccess && p->precision == ES_PREC_MIXED) e = d3f_prepare();
        }
        else e = p->precision == ES_PREC_MIXED ? stage_prepare_mixed(p->dim) : stage_prepare_fp64(p->dim);
        if (e != cudaSuccess) { rc = cuda_fail(c, e, "stage kernel attributes"); goto fail_out; }
    }
    if (p->dim == 3) {
        c->d3 = (Ctx3*)calloc(1, sizeof(Ctx3));
        if (!c->d3) { rc = fail(c, ES_ERR_ARG, "out of host memory"); goto fail_out; }
        Ctx3* d = c->d3;
        const int nn[3] = {p->n1, p->n2, p->n3};
        for (int k = 0; k < 3; ++k) {
            d->g.n[k] = nn[k];
            d->g.bc[k] = p->bc[k];
            d->g.inv_dxi[k] = 1.0 / p->dxi[k];
            d->g.finv[k] = float(d->g.inv_dxi[k]);
            d->g.finv2[k] = float(d->g.inv_dxi[k] * d->g.inv_dxi[k]);
            d->g.period[k] = p->period[k];
        }
        d->gas = c->gas;
        d->weno = c->weno;
        d->mon = c->mon;
        d->diss = p->dissipation;
        d->mixed = c->mixed;
        d->filter_passes = p->filter_passes;
        d->sweeps = p->jacobi_sweeps;
        d->eps = p->jacobi_eps;
        const size_t blocks = (c->N + 255) / 256;             // 256-thread grid-stride kernels
        d->grid = (int)(blocks < size_t(nsm) * 8 ? blocks : size_t(nsm) * 8);
        // tile 0: chosen by es_autotune; mixed tiles D3_NSHAPES + k: shape k with plain loads (no TMA staging)
        d->shape = p->tile >= 1 ? (p->tile - 1) % D3_NSHAPES : 0;
        d->no_tma = p->tile > D3_NSHAPES;
        d->rhoF = c->rhoF;
        d->GF = c->GF;
        d->t0 = c->t0;
        d->t1 = c->t1;
        d->t2 = c->t2;
        d->om0 = c->om0;
        d->om1 = c->om1;
        d->xa = c->xa;
        d->xb = c->xb;
        d->gc = c->fdisp;                  // [3][N] floats, allocated for the mixed form
        cudaError_t e = d3_alloc(d);
        if (e != cudaSuccess) { rc = cuda_fail(c, e, "cudaMalloc (3D scratch)"); goto fail_out; }
    }
    *out = c;
    return ES_OK;
fail_out:
    es_destroy(c);
    return rc;
}

void es_destroy(es_ctx* c) {
    if (!c) return;
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->body_stream) cudaStreamDestroy(c->body_stream);
    void* bufs[] = {c->S1, c->S2, c->S1J, c->S2J, c->rhoF, c->GF, c->t0, c->t1, c->t2, c->om0, c->om1,
                    c->xa, c->xb, c->xdot, c->hJU, c->hJ, c->hx, c->fdisp, c->fxd,
                    c->nn_wbf, c->nn_b, c->feat, c->act0, c->act1, c->nn_out, c->xw};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (c->dev) cudaFree(c->dev);
    if (c->hpin) cudaFreeHost(c->hpin);
    if (c->d3) {
        d3_free(c->d3);
        free(c->d3);
    }
    free(c);
}

int es_init_mesh(es_ctx* c, const double* x, void* J) {
    if (!c || !x || !J) return fail(c, ES_ERR_ARG, "null argument");
    if (c->d3) {
        cudaError_t e;
        if (d3_init_J(c->d3, x, (double*)J, c->stream, &e) < 0) return cuda_fail(c, e, "k3_init_J");
        count(c);
        return ES_OK;
    }
    launch_init_J(c->g, x, J, c->mixed, c->grid1d, c->stream);
    count(c);
    CK(cudaGetLastError(), "k_init_J");
    return ES_OK;
}

int es_prim_to_cons(es_ctx* c, const double* rho, const double* v, const double* p, const void* J, void* JU) {
    if (!c || !rho || !v || !p || !J || !JU) return fail(c, ES_ERR_ARG, "null argument");
    launch_prim_to_cons(c->g, c->gas, rho, v, p, J, JU, c->mixed, c->grid1d, c->stream);
    count(c);
    CK(cudaGetLastError(), "k_prim_to_cons");
    return ES_OK;
}

int es_rhs(es_ctx* c, const void* JU, const void* J, const double* x, const double* xdot, void* dJU, void* dJ) {
    if (!c || !JU || !J || !x || !dJU || !dJ) return fail(c, ES_ERR_ARG, "null argument");
    if (c->d3) {
        Stage3 a = {};
        a.JUn = a.JUs = (const double*)JU;
        a.Jn = a.Js = (const double*)J;
        a.xn = x;
        a.xdot = xdot;
        a.JUo = (double*)dJU;
        a.Jo = (double*)dJ;
        a.dt_host = 1.0;
        a.mode = 1;
        cudaError_t e;
        const int n = d3_stage(c->d3, a, &c->dev->status, c->stream, &e);
        if (n < 0) return cuda_fail(c, e, "3D stage kernels");
        count(c, n);
        return ES_OK;
    }
    StageParams P = stage_params(c);
    P.mode = 1;
    P.dt_host = 1.0;
    P.xn = x;
    P.xdot = xdot;
    enqueue_mesh_f32(c, P, x, xdot);
    set_state(c, P, JU, J, JU, J, dJU, dJ);
    CK(launch_stage(c, P), "stage kernel");
    return ES_OK;
}

int es_rk_stage(es_ctx* c, int stage, double dt, const void* JUn, const void* Jn, const void* JUs,
                const void* Js, const double* xn, const double* xdot, void* JU_out, void* J_out) {
    if (!c || stage < 1 || stage > 3 || !JUn || !Jn || !JUs || !Js || !xn || !JU_out || !J_out)
        return fail(c, ES_ERR_ARG, "bad argument");
    if (JU_out == JUs || J_out == Js) return fail(c, ES_ERR_ARG, "output aliases the stage input");
    if (c->d3) {
        Stage3 a = {};
        a.JUn = (const double*)JUn;
        a.Jn = (const double*)Jn;
        a.JUs = (const double*)JUs;
        a.Js = (const double*)Js;
        a.xn = xn;
        a.xdot = xdot;
        a.JUo = (double*)JU_out;
        a.Jo = (double*)J_out;
        a.ca = RK_A[stage - 1];
        a.cb = RK_B[stage - 1];
        a.cst = RK_C[stage - 1];
        a.dt_host = dt;
        a.mode = 0;
        cudaError_t e;
        const int n = d3_stage(c->d3, a, &c->dev->status, c->stream, &e);
        if (n < 0) return cuda_fail(c, e, "3D stage kernels");
        count(c, n);
        return ES_OK;
    }
    StageParams P = stage_params(c);
    P.ca = RK_A[stage - 1];
    P.cb = RK_B[stage - 1];
    P.cst = RK_C[stage - 1];
    P.dt_host = dt;
    P.xn = xn;
    P.xdot = xdot;
    enqueue_mesh_f32(c, P, xn, xdot);
    set_state(c, P, JUn, Jn, JUs, Js, JU_out, J_out);
    CK(launch_stage(c, P), "stage kernel");
    return ES_OK;
}

int es_cfl_dt(es_ctx* c, const void* JU, const void* J, const double* x, const double* xdot, double* dt_host) {
    if (!c || !JU || !J || !x || !dt_host) return fail(c, ES_ERR_ARG, "null argument");
    const int slot = xdot ? RED_CFL2 : RED_CFL;
    k_reset<<<1, 32, 0, c->stream>>>(c->dev);
    count(c);
    if (c->d3) {
        cudaError_t e;
        int n = d3_cfl(c->d3, (const double*)JU, (const double*)J, x, c->dev, c->stream, &e);
        if (n >= 0 && xdot) n = d3_cfl_moving(c->d3, J, xdot, c->dev, c->stream, &e);
        if (n < 0) return cuda_fail(c, e, "3D time-step kernels");
        count(c, n);
    } else if (mesh_on_fp32(c)) {
        k_mesh_f32<<<c->grid1d, c->block1d, 0, c->stream>>>(c->g, x, xdot, c->fdisp, c->fxd);
        k_cfl_f<<<c->grid1d, c->block1d, 0, c->stream>>>(c->g, gas_f32(c->gas), (const float*)JU, (const float*)J,
                                                   c->fdisp, xdot ? c->fxd : nullptr, slot, c->dev);
        count(c, 2);
    } else {
        enqueue_cfl(c, JU, J, x, xdot, slot);
    }
    CK(cudaGetLastError(), "k_cfl");
    CK(cudaMemcpyAsync(c->hpin, c->dev, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "sync");
    double mx;
    memcpy(&mx, &c->hpin->red[slot], sizeof(double));
    *dt_host = c->p.cfl / mx;
    return ES_OK;
}

int es_entropy_rate(es_ctx* c, const void* JU, const void* J, const void* dJU, const void* dJ, double* out_host) {
    if (!c || !JU || !J || !dJU || !dJ || !out_host) return fail(c, ES_ERR_ARG, "null argument");
    double vol = 1.0;
    for (int k = 0; k < c->p.dim; ++k) vol *= c->p.dxi[k];
    // t0 (per-block partial sums, 3 per block <= the mesh size) and t1 (the result) are mesh-solve scratch
    launch_entropy_rate(int(c->N), c->p.dim, c->gas, JU, J, dJU, dJ, vol, c->t0, c->t1, c->mixed, c->grid1d,
                        c->stream);
    count(c, 2);
    CK(cudaGetLastError(), "entropy kernels");
    CK(cudaMemcpyAsync(c->hpin->last_change, c->t1, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "sync");
    out_host[0] = c->hpin->last_change[0];
    out_host[1] = c->hpin->last_change[1];
    return ES_OK;
}

int es_mesh_redistribute(es_ctx* c, const void* JU, const void* J, const double* xn, double dt,
                         double* xdot, int* sweeps_host, double* gamma_host) {
    if (!c || !JU || !J || !xn || !xdot || !(dt > 0.0)) return fail(c, ES_ERR_ARG, "bad argument");
    k_reset<<<1, 32, 0, c->stream>>>(c->dev);
    k_set_dt<<<1, 32, 0, c->stream>>>(c->dev, dt);
    count(c, 2);
    int rc;
    if (c->d3) {
        cudaError_t e;
        const int n = d3_mesh(c->d3, (const double*)JU, (const double*)J, xn, xdot, c->dev, c->stream, &e);
        if (n < 0) return cuda_fail(c, e, "3D mesh kernels");
        count(c, n);
        rc = ES_OK;
    } else if (mesh_on_fp32(c)) {
        k_mesh_f32<<<c->grid1d, c->block1d, 0, c->stream>>>(c->g, xn, nullptr, c->fdisp, c->fxd);
        count(c);
        rc = enqueue_mesh32(c, JU, J, xdot, 0);
    } else {
        rc = enqueue_mesh(c, JU, J, xn, xdot);
    }
    if (rc) return rc;
    if (sweeps_host || gamma_host) {
        CK(cudaMemcpyAsync(c->hpin, c->dev, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream), "copy");
        CK(cudaStreamSynchronize(c->stream), "sync");
        if (sweeps_host) *sweeps_host = c->hpin->sweeps;
        if (gamma_host) *gamma_host = c->hpin->gamma;
    }
    return ES_OK;
}

int es_mesh_features(es_ctx* c, const void* JU, const void* J, const double* x, float* feat) {
    if (!c || !JU || !J || !x || !feat) return fail(c, ES_ERR_ARG, "null argument");
    if (c->p.dim != 2) return fail(c, ES_ERR_ARG, "features are defined for 2D meshes");
    k_reset<<<1, 32, 0, c->stream>>>(c->dev);
    count(c);
    const double* om = enqueue_monitor(c, JU, J);
    k_features<<<c->grid1d, c->block1d, 0, c->stream>>>(c->g, om, c->GF, x, feat);
    count(c);
    CK(cudaGetLastError(), "feature kernels");
    return ES_OK;
}

int es_mesh_solve(es_ctx* c, const void* JU, const void* J, const double* xn, const double* x_start,
                  double guard_ratio, double* x_out, float* disp_out, int* sweeps_host, int* picked_host) {
    if (!c || !JU || !J || !xn || (!x_out && !disp_out)) return fail(c, ES_ERR_ARG, "null argument");
    if (x_out && (x_out == xn || (x_start && x_out == x_start))) return fail(c, ES_ERR_ARG, "x_out aliases an input");
    if (x_start && !(guard_ratio >= 0.0)) return fail(c, ES_ERR_ARG, "guard ratio must be >= 0");
    if (c->d3) return fail(c, ES_ERR_ARG, "es_mesh_solve is defined for 1D and 2D meshes");
    k_reset<<<1, 32, 0, c->stream>>>(c->dev);
    count(c);
    const double* om = enqueue_monitor(c, JU, J);
    const int rj = enqueue_jacobi(c, om, xn, x_start, guard_ratio);
    if (rj) return rj;
    k_jacobi_out<<<c->grid1d, c->block1d, 0, c->stream>>>(c->g, xn, c->xa, c->xb, c->dev, x_out, disp_out);
    count(c);
    CK(cudaGetLastError(), "mesh kernels");
    if (sweeps_host || picked_host) {
        CK(cudaMemcpyAsync(c->hpin, c->dev, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream), "copy");
        CK(cudaStreamSynchronize(c->stream), "sync");
        if (sweeps_host) *sweeps_host = c->hpin->sweeps;
        if (picked_host) *picked_host = c->hpin->pick;
    }
    return ES_OK;
}

int es_mesh_warm_start(es_ctx* c, const double* xn, const float* out, double* x_start) {
    if (!c || !xn || !out || !x_start) return fail(c, ES_ERR_ARG, "null argument");
    if (c->p.dim != 2) return fail(c, ES_ERR_ARG, "the warm start is defined for 2D meshes");
    if (x_start == xn) return fail(c, ES_ERR_ARG, "x_start aliases xn");
    k_warm_start<<<c->grid1d, c->block1d, 0, c->stream>>>(c->g, xn, out, x_start);
    count(c);
    CK(cudaGetLastError(), "k_warm_start");
    return ES_OK;
}

int es_set_warm_start(es_ctx* c, const uint16_t* w_bf16, const float* bias, int layers, int hidden,
                      double guard_ratio) {
    if (!c) return ES_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream), "sync");
    drop_graphs(c);                        // the step graphs change with the network
    if (!w_bf16) {
        c->nn_layers = 0;
        return ES_OK;
    }
    if (!bias || c->p.dim != 2 || layers < 2 || layers > 16 || !(hidden == 4 || hidden == 32) ||
        !(guard_ratio >= 0.0))
        return fail(c, ES_ERR_ARG, "warm start: 2D only, 2..16 layers, hidden 4 or 32, guard ratio >= 0");
    const int cin0 = c->p.dim + 2;
    const size_t nw = size_t(hidden) * cin0 * 9 + size_t(layers - 2) * hidden * hidden * 9 +
                      size_t(c->p.dim) * hidden * 9;
    const size_t nb = size_t(layers - 1) * hidden + c->p.dim;
    if (c->nn_hidden != hidden || !c->feat) {
        void* old[] = {c->nn_b, c->act0, c->act1};
        for (void* b : old)
            if (b) cudaFree(b);
        c->nn_b = c->act0 = c->act1 = nullptr;
        const size_t FB = sizeof(float) * c->N;
        if (!c->feat) {
            CK(cudaMalloc((void**)&c->feat, FB * cin0), "cudaMalloc");
            CK(cudaMalloc((void**)&c->nn_out, FB * c->p.dim), "cudaMalloc");
            CK(cudaMalloc((void**)&c->xw, sizeof(double) * c->N * c->p.dim), "cudaMalloc");
        }
        CK(cudaMalloc((void**)&c->act0, FB * hidden), "cudaMalloc");
        CK(cudaMalloc((void**)&c->act1, FB * hidden), "cudaMalloc");
    }
    if (c->nn_wbf) cudaFree(c->nn_wbf);
    if (c->nn_b) cudaFree(c->nn_b);
    c->nn_wbf = nullptr;
    c->nn_b = nullptr;
    CK(cudaMalloc((void**)&c->nn_wbf, sizeof(uint16_t) * nw), "cudaMalloc");
    CK(cudaMalloc((void**)&c->nn_b, sizeof(float) * nb), "cudaMalloc");
    CK(cudaMemcpyAsync(c->nn_wbf, w_bf16, sizeof(uint16_t) * nw, cudaMemcpyDeviceToDevice, c->stream), "weight copy");
    CK(cudaMemcpyAsync(c->nn_b, bias, sizeof(float) * nb, cudaMemcpyDeviceToDevice, c->stream), "bias copy");
    CK(nn_prepare(), "conv kernel attributes");
    CK(cudaStreamSynchronize(c->stream), "sync");
    c->nn_layers = layers;
    c->nn_hidden = hidden;
    c->nn_ratio = guard_ratio;
    return ES_OK;
}

int es_mesh_stats(es_ctx* c, int64_t* sweeps_total, int64_t* solves, int64_t* warm_kept, int reset) {
    if (!c) return ES_ERR_ARG;
    CK(cudaMemcpyAsync(c->hpin, c->dev, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (sweeps_total) *sweeps_total = c->hpin->sweeps_total;
    if (solves) *solves = c->hpin->solves;
    if (warm_kept) *warm_kept = c->hpin->warm_kept;
    if (reset) {
        c->hpin->sweeps_total = c->hpin->solves = c->hpin->warm_kept = 0;
        const size_t off = offsetof(DevScalars, sweeps_total);
        CK(cudaMemcpyAsync((char*)c->dev + off, (char*)c->hpin + off, 3 * sizeof(long long),
                           cudaMemcpyHostToDevice, c->stream), "copy");
        CK(cudaStreamSynchronize(c->stream), "sync");
    }
    return ES_OK;
}

int es_set_time(es_ctx* c, double t) {
    if (!c) return ES_ERR_ARG;
    CK(cudaMemcpyAsync(c->hpin, c->dev, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "sync");
    c->hpin->t = t;
    c->hpin->last_dt = 0.0;
    CK(cudaMemcpyAsync(c->dev, c->hpin, sizeof(DevScalars), cudaMemcpyHostToDevice, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "sync");
    return ES_OK;
}

int es_get_time(es_ctx* c, double* t_host, double* last_dt_host) {
    if (!c) return ES_ERR_ARG;
    CK(cudaMemcpyAsync(c->hpin, c->dev, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (t_host) *t_host = c->hpin->t;
    if (last_dt_host) *last_dt_host = c->hpin->last_dt;
    return ES_OK;
}

int es_step(es_ctx* c, void* JU, void* J, double* x, double t_end, double* t_host, double* dt_host) {
    const int rc = es_steps(c, JU, J, x, 1, t_end);
    if (rc || (!t_host && !dt_host)) return rc;
    return es_get_time(c, t_host, dt_host);
}

// one step captured into an executable graph on the private capture stream
static int capture_step(es_ctx* c, void* JU, void* J, double* x, bool first, bool chain, cudaGraphExec_t* out,
                        int* kernels) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    c->capturing = 1;
    c->capture_count = 0;
    c->s_enq = c->cap_stream;
    int rc = enqueue_step(c, JU, J, x, first, chain);
    c->s_enq = c->stream;
    c->capturing = 0;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (rc) {
        if (e == cudaSuccess && graph) cudaGraphDestroy(graph);    // never instantiated
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    *kernels = c->capture_count;
    return ES_OK;
}

int es_steps(es_ctx* c, void* JU, void* J, double* x, int nsteps, double t_end) {
    if (!c || !JU || !J || !x || nsteps < 0) return fail(c, ES_ERR_ARG, "bad argument");
    if (nsteps == 0) return ES_OK;
    // t_end lives on the device: a one-thread kernel writes it, ordered on the stream, when it changes (a copy from
    // pinned host memory needed a synchronisation before the buffer could be reused, and that left the GPU idle
    // between the caller's previous work and the steps)
    if (!(c->t_end_dev == t_end)) {
        k_set_t_end<<<1, 32, 0, c->stream>>>(c->dev, t_end);
        count(c);
        CK(cudaGetLastError(), "t_end kernel");
        c->t_end_dev = t_end;
    }
    if (!c->tuned) {
        int rc = es_autotune(c, JU, J, x, nullptr, nullptr);
        if (rc) return rc;
    }
    const void* key[3] = {JU, J, x};
    if (memcmp(key, c->gkey, sizeof(key)) != 0) {
        drop_graphs(c);
        memcpy(c->gkey, key, sizeof(key));
    }
    const int first = nsteps == 1 ? 0 : 1;
    for (int k = first; k <= (nsteps == 1 ? 0 : 2); ++k) {
        if (!c->gexec[k]) {
            int rc = capture_step(c, JU, J, x, k < 2, k > 0, &c->gexec[k], &c->graph_kernels[k]);
            if (rc) return rc;
        }
    }
    for (int k = 0; k < nsteps; ++k) {
        const int g = k == 0 ? first : 2;
        CK(cudaGraphLaunch(c->gexec[g], c->stream), "graph launch");
        c->launches += c->graph_kernels[g];
    }
    return ES_OK;
}

int es_run_host(es_ctx* c, void* JU_host, void* J_host, double* x_host, int nsteps, double t_end) {
    if (!c || !JU_host || !J_host || !x_host) return fail(c, ES_ERR_ARG, "null argument");
    const size_t SB = c->esz * c->N;
    const size_t XB = sizeof(double) * c->N * c->p.dim;
    if (!c->hJU) {
        CK(cudaMalloc(&c->hJU, SB * c->nc), "cudaMalloc");
        CK(cudaMalloc(&c->hJ, SB), "cudaMalloc");
        CK(cudaMalloc((void**)&c->hx, XB), "cudaMalloc");
    }
    CK(cudaMemcpyAsync(c->hJU, JU_host, SB * c->nc, cudaMemcpyHostToDevice, c->stream), "h2d");
    CK(cudaMemcpyAsync(c->hJ, J_host, SB, cudaMemcpyHostToDevice, c->stream), "h2d");
    CK(cudaMemcpyAsync(c->hx, x_host, XB, cudaMemcpyHostToDevice, c->stream), "h2d");
    int rc = es_steps(c, c->hJU, c->hJ, c->hx, nsteps, t_end);
    if (rc) return rc;
    CK(cudaMemcpyAsync(JU_host, c->hJU, SB * c->nc, cudaMemcpyDeviceToHost, c->stream), "d2h");
    CK(cudaMemcpyAsync(J_host, c->hJ, SB, cudaMemcpyDeviceToHost, c->stream), "d2h");
    CK(cudaMemcpyAsync(x_host, c->hx, XB, cudaMemcpyDeviceToHost, c->stream), "d2h");
    CK(cudaStreamSynchronize(c->stream), "sync");
    return ES_OK;
}

// 3D: time the operator (metrics, node fields, three direction launches) with each pencil shape
static int autotune3(es_ctx* c, const void* JU, const void* J, const double* x, int* tile_host, double* ms_host) {
    CK(cudaStreamSynchronize(c->stream), "sync");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(c, e, "event");
    }
    Stage3 a = {};
    a.JUn = a.JUs = (const double*)JU;
    a.Jn = a.Js = (const double*)J;
    a.xn = x;
    a.JUo = (double*)c->S1;
    a.Jo = (double*)c->S1J;
    a.dt_host = 1.0;
    a.mode = 1;
    const int saved = c->d3->shape;
    int best = 0;
    float best_ms = 3.0e38f;
    for (int k = 0; k < D3_NSHAPES && e == cudaSuccess; ++k) {
        c->d3->shape = k;
        float ms = 0.0f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {   // the first evaluation loads the kernels
            e = cudaEventRecord(e0, c->stream);
            if (e == cudaSuccess) {
                cudaError_t el;
                const int n = d3_stage(c->d3, a, &c->dev->status, c->stream, &el);
                if (n < 0) e = el;
                else count(c, n);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t;
        }
        if (ms_host) ms_host[k] = ms / 2;
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        c->d3->shape = saved;
        return cuda_fail(c, e, "autotune");
    }
    c->d3->shape = best;
    c->tuned = 1;
    drop_graphs(c);                        // the step graphs hold the old shape
    if (tile_host) *tile_host = best + 1;
    return ES_OK;
}

int es_autotune(es_ctx* c, const void* JU, const void* J, const double* x, int* tile_host, double* ms_host) {
    if (!c || !JU || !J || !x) return fail(c, ES_ERR_ARG, "null argument");
    if (c->p.dim == 1) {                 // one stage shape in 1D
        c->tuned = 1;
        if (tile_host) *tile_host = 1;
        return ES_OK;
    }
    if (c->d3) return autotune3(c, JU, J, x, tile_host, ms_host);
    CK(cudaStreamSynchronize(c->stream), "sync");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(c, e, "event");
    }
    int best = 0;
    float best_ms = 3.0e38f;
    const int saved = c->tile;
    for (int k = 0; k < ES_NTILES && e == cudaSuccess; ++k) {
        c->tile = k;
        StageParams P = stage_params(c);
        P.mode = 1;
        P.dt_host = 1.0;
        P.xn = x;
        P.xdot = nullptr;
        enqueue_mesh_f32(c, P, x, nullptr);
        set_state(c, P, JU, J, JU, J, c->S1, c->S1J);
        float ms = 0.0f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {   // the first launch loads the kernel
            e = cudaEventRecord(e0, c->stream);
            if (e == cudaSuccess) e = launch_stage(c, P);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t;
        }
        if (ms_host) ms_host[k] = ms / 2;
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        c->tile = saved;
        return cuda_fail(c, e, "autotune");
    }
    c->tile = best;
    c->tuned = 1;
    drop_graphs(c);                        // the step graphs hold the old shape
    if (tile_host) *tile_host = best + 1;
    return ES_OK;
}

int es_time_stage(es_ctx* c, const void* JU, const void* J, const double* x, int stage, double dt, int reps,
                  double* ms_host) {
    if (!c || !JU || !J || !x || !ms_host || stage < 1 || stage > 3 || reps < 1 || !(dt > 0.0))
        return fail(c, ES_ERR_ARG, "bad argument");
    if (c->d3) return fail(c, ES_ERR_ARG, "es_time_stage: 1D/2D contexts only");
    StageParams P = stage_params(c);
    P.ca = RK_A[stage - 1];
    P.cb = RK_B[stage - 1];
    P.cst = RK_C[stage - 1];
    P.dt_host = dt;
    P.xn = x;
    P.xdot = nullptr;
    enqueue_mesh_f32(c, P, x, nullptr);
    set_state(c, P, JU, J, JU, J, c->S1, c->S1J);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(c, e, "event");
    }
    e = launch_stage(c, P);                                  // loads the kernel before the timed launches
    if (e == cudaSuccess) e = cudaEventRecord(e0, c->s_enq);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_stage(c, P);
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->s_enq);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "es_time_stage");
    *ms_host = double(ms) / reps;
    return ES_OK;
}

int es_check(es_ctx* c) {
    if (!c) return ES_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream), "sync");
    CK(cudaMemcpy(c->hpin, c->dev, sizeof(DevScalars), cudaMemcpyDeviceToHost), "copy status");
    const int code = c->hpin->status.code;
    if (code != ES_OK) {
        const char* what = code == ES_ERR_INADMISSIBLE ? "inadmissible state (eq. coefflimit / Theorem 3.1)"
                         : code == ES_ERR_MESH         ? "non-positive J (mesh folded)"
                         : code == ES_ERR_TIMEOUT      ? "device wait timed out"
                                                       : "device error";
        snprintf(c->msg, sizeof(c->msg), "%s at node %d", what, c->hpin->status.index);
        DevStatus z = {0, 0};
        CK(cudaMemcpy(&c->dev->status, &z, sizeof(z), cudaMemcpyHostToDevice), "clear status");
    }
    return code;
}

int es_last_error(es_ctx* c, char* buf, int len) {
    if (!c || !buf || len <= 0) return ES_ERR_ARG;
    snprintf(buf, len, "%s", c->msg);
    return ES_OK;
}

int64_t es_launch_count(es_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
