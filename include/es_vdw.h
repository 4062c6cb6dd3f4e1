/*
 * es_vdw.h -- C ABI of the GB300 (sm_103a) library for the high-order
 * entropy-stable finite-difference scheme for the Euler equations with the
 * van der Waals equation of state on an adaptive moving mesh
 * (Li & Tang, arXiv:2407.05568).
 *
 * Data layout (all calls)
 *   Node-centred fields on a logically rectangular n1 x n2 mesh (n2 = 1 in 1D),
 *   structure of arrays, xi_1 fastest:  field[c][j][i] at c*n1*n2 + j*n1 + i;
 *   in 3D an n1 x n2 x n3 mesh, field[c][k][j][i] at ((c*n3 + k)*n2 + j)*n1 + i.
 *     JU : (dim + 2) components (rho, rho v_1, [rho v_2, [rho v_3]], E) times J
 *     J  : 1 component
 *     JU, J (and dJU, dJ) hold double in ES_PREC_FP64.  In ES_PREC_MIXED they
 *     hold compensated float pairs in two planes: [2][dim+2][n2][n1] for JU and
 *     [2][n2][n1] for J, value = hi plane + lo plane (a 48-bit significand in
 *     8 bytes, like a double).  They are passed as void*.
 *     x  : dim components (x_1, [x_2, [x_3]]) of the node coordinates, double
 *     xdot : dim components of the mesh velocity, double
 *   The computational mesh is uniform with spacings dxi[k]; x(xi) maps it to
 *   the physical mesh (Sec. 3, eq. transf).
 *
 * Three dimensions (dim = 3)
 *   The operator, the SSP-RK3 stages and the mesh redistribution in their 3D form:
 *   the cross-form metrics of Sec. 3.2 (eq. SCLCoeff), the theta/phi rotation of
 *   Sec. 3.3 and the 27-point filter of Sec. 4, in both precision forms (the mixed
 *   form: FP32 direction kernels, double-float metrics and state; walls and symmetry
 *   planes in ES_PREC_FP64 only).  es_create,
 *   es_init_mesh, es_prim_to_cons, es_rhs, es_rk_stage, es_cfl_dt,
 *   es_mesh_redistribute, es_steps, es_run_host, es_autotune (four pencil shapes) and the
 *   time and status calls accept a 3D context; es_mesh_features, es_mesh_solve,
 *   es_mesh_warm_start and es_set_warm_start return ES_ERR_ARG for it.  A 3D
 *   context holds about 66 n1 n2 n3 + 12 (n1+6)(n2+6)(n3+6) doubles of scratch.
 *
 * Pointers
 *   Every array argument is a DEVICE pointer (cudaMalloc'd or a PyTorch
 *   tensor's storage) owned by the caller, except where a name ends in _host.
 *   The library never frees caller memory.  The context owns its scratch.
 *
 * Streams and errors
 *   Calls are asynchronous on the context's stream.  The return value reports
 *   argument and launch errors only (ES_OK = 0).  Errors found on the device
 *   (an inadmissible state, a folded mesh) latch in a device word read by
 *   es_check(), which synchronises the stream.  es_last_error() gives the text.
 */
#ifndef ES_VDW_H
#define ES_VDW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ES_OK               0
#define ES_ERR_ARG          1   /* bad argument (size, null pointer, unsupported option) */
#define ES_ERR_CUDA         2   /* a CUDA runtime call failed */
#define ES_ERR_INADMISSIBLE 3   /* eq. coefflimit / Theorem 3.1 violated at some node or face */
#define ES_ERR_MESH         4   /* J <= 0 or the mesh folded */
#define ES_ERR_TIMEOUT      5   /* a bounded device wait ran out */

/* boundary conditions, per direction */
#define ES_BC_PERIODIC 0        /* wrap; coordinates shifted by period[k] */
#define ES_BC_OUTFLOW  1        /* state copied; coordinates reflected; boundary nodes fixed */
#define ES_BC_REFLECT  2        /* wall at both ends (ES_PREC_FP64 only): the mirror image about the
                                   boundary node -- state mirrored with the normal momentum negated,
                                   coordinates and mesh velocity mirrored along the wall and reflected
                                   across it; boundary nodes slide along the wall */
#define ES_BC_SYMMETRY_LO 3     /* symmetry plane at the low end as ES_BC_REFLECT, outflow at the high
                                   end (ES_PREC_FP64 only; e.g. an octant of a spherical problem) */

/* arithmetic of the operator */
#define ES_PREC_FP64   0        /* every step in double */
#define ES_PREC_MIXED  1        /* per-stage arithmetic on the FP32 pipe: the state and the primitive
                                   variables in double-float (hi + lo float pairs), fluxes and WENO in
                                   float, entropy-variable jumps by the paper's jump decomposition, the
                                   mesh as an FP32 displacement from the Cartesian mesh; the CFL step and
                                   the mesh redistribution also run on that displacement in float (with a
                                   warm-start network registered they use the double kernels); the mesh x
                                   itself stays double.  Periodic directions need period[k] = n_k dxi[k]. */

/* monitor functions of Sec. 4 / Example 5.1 */
#define ES_MONITOR_VDW    0     /* eq. van der Waalsmonitor: delta_1 = rho, delta_2 = G, plus |Delta G|^2 */
#define ES_MONITOR_SMOOTH 1     /* eq. van der Waalssinmonitor: |grad rho| and |Delta rho| */

typedef struct es_params {
    /* van der Waals gas, Sec. 1 eq. vdWEOS: p = rho R T/(1 - b rho) - a rho^2, e = cv T - a rho.
       a = b = 0 is the ideal gas. */
    double a, b, R, cv;
    int    dim;             /* 1, 2 or 3 */
    int    n1, n2, n3;      /* nodes per direction, each >= 8 in use; n2 = 1 when dim = 1; n3 = 0 or 1
                               when dim < 3 */
    double dxi[3];          /* computational spacings Delta xi_k */
    double period[3];       /* period of x_k along a periodic direction */
    int    bc[3];           /* ES_BC_* per direction */
    double weno_gamma[3];   /* MR-WENO5 linear weights (1-point, 3-point, 5-point), Sec. 5: (0.005, 0.045, 0.95) */
    double weno_eps;        /* epsilon of the MR-WENO5 nonlinear weights (paper silent; 1e-6, Jiang and Shu's) */
    double sign_tol;        /* sign switch Y: a plain jump |W_{i+1} - W_i| no larger than sign_tol times
                               sum_a |R_am| (|(TV_i)_a| + |(TV_{i+1})_a|), the size of the terms forming
                               it, is round-off of a zero jump and has sign 0 (Y = 0): 1e-12 in
                               ES_PREC_FP64, 4e-7 (a few FP32 roundings) in ES_PREC_MIXED */
    int    dissipation;     /* 1: ES flux eq. HOstable; 0: the EC flux alone */
    double cfl;             /* eq. cfl; 0.4 in 1D/2D */
    double dt_fixed;        /* > 0: use this Delta t instead of eq. cfl (Example 5.1 uses CFL dxi^(5/3)) */
    int    moving;          /* 1: adaptive moving mesh (Sec. 4) */
    int    monitor;         /* ES_MONITOR_* */
    int    kappa;           /* number of gradient terms of the vdW monitor (1: rho; 2: rho and G) */
    double alpha[4];        /* monitor weights alpha_1 .. alpha_{kappa+1} */
    int    filter_passes;   /* low-pass filter passes (Sec. 4) */
    int    jacobi_sweeps;   /* mu: maximum Jacobi sweeps (Sec. 4) */
    double jacobi_eps;      /* stop when max |x^[nu+1] - x^[nu]| < eps; 0 = exactly mu sweeps */
    int    precision;       /* ES_PREC_* */
    int    tile;            /* stage tile shape: 0 = chosen by es_autotune (run by the first es_steps
                               if not called before); k = 1 .. ES_NTILES: shape k of the precision's
                               2D table (FP64: 32x8, 25x11, 16x16, 32x12, 20x10 nodes; mixed: 20x8 with two
                               lanes per face, 25x6, 20x8, 16x8 with two lanes per face, 16x8); in 3D the
                               direction kernels' pencils, FP64:
                               1 = 16 nodes x 16 lines, 2 = 16 x 8, 3 = 16 x 4, 4 = 32 x 4; mixed:
                               1 = 16 x 16, 2 = 32 x 8, 3 = 16 x 8, 4 = 32 x 4, and 5 .. 8 the same
                               shapes with node-by-node loads instead of the TMA staging of the xi_2 and
                               xi_3 pencils (which needs n1 a multiple of 4) */
} es_params;

#define ES_NTILES 5

typedef struct es_ctx es_ctx;

/* Create a context for one mesh size and parameter set on the current device.
 * stream: a cudaStream_t (NULL = legacy default stream).  Allocates the
 * scratch it needs (a few fields of the mesh size).  Returns ES_ERR_ARG for
 * unsupported sizes or options. */
int es_create(es_ctx** ctx, const es_params* p, void* stream);
void es_destroy(es_ctx* ctx);

/* Initial metric Jacobian J = det dx/dxi at the nodes, from the same 6th-order
 * central differences delta_k used by the metrics (Sec. 3.2, eq. SCLCoeff).
 * x: [dim][n2][n1] in, J: [n2][n1] out. */
int es_init_mesh(es_ctx* ctx, const double* x, void* J);

/* Conservative variables JU = J (rho, rho v, E) from primitive (rho, v, p)
 * (Sec. 1, eq. ConserLaw2 with E = rho e + rho |v|^2/2, T from eq. vdWEOS).
 * rho, p: [n2][n1]; v: [dim][n2][n1]; J: [n2][n1]; JU out: [dim+2][n2][n1]. */
int es_prim_to_cons(es_ctx* ctx, const double* rho, const double* v, const double* p,
                    const void* J, void* JU);

/* Semi-discrete operator alone (eq. semi_U, eq. semi_J):
 *   dJU = -sum_k (F_{k,+1/2} - F_{k,-1/2}) / dxi_k,  dJ likewise with the J xi_t fluxes,
 * with the 6th-order EC flux (eq. ECFlux_curv_2p, GCL_flux), the metrics of the
 * mesh x moving with velocity xdot (eq. SCLCoeff, VCLCoeff) and, when
 * p->dissipation, the ES dissipation (eq. HOstable).  All device arrays. */
int es_rhs(es_ctx* ctx, const void* JU, const void* J, const double* x, const double* xdot,
           void* dJU, void* dJ);

/* One SSP-RK3 stage (Shu-Osher form, stage = 1, 2, 3):
 *   (JU, J)_out = a_s (JU, J)_n + b_s ((JU, J)_s + dt L(JU_s, J_s; x_s)),
 * (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3); the operator is evaluated on the stage
 * mesh x_s = xn + c_s dt xdot with c = (0, 1, 1/2).  JUn/Jn are read only at the
 * node itself, so JU_out may alias JUn (but not JUs). */
int es_rk_stage(es_ctx* ctx, int stage, double dt,
                const void* JUn, const void* Jn, const void* JUs, const void* Js,
                const double* xn, const double* xdot, void* JU_out, void* J_out);

/* Time step of eq. cfl (Sec. 5): CFL / max_i sum_k (|J xi_{k,t} + n_k . v| + |n_k| c) / (J dxi_k), the
 * spectral radius of the xi_k flux Jacobian with J xi_{k,t} = -xdot . n_k (eq. VCLCoeff).  xdot is the
 * mesh velocity [dim][n...] (device, double) or NULL for a mesh at rest.  Synchronises the context's
 * stream and writes the host double. */
int es_cfl_dt(es_ctx* ctx, const void* JU, const void* J, const double* x, const double* xdot, double* dt_host);

/* Entropy production check in FP64 (Sec. 2-3): the rate of the total entropy sum_i J_i eta(U_i) dV,
 *   out_host[0] = dV sum_i (V_i . dJU_i - phi_i dJ_i),   out_host[1] = dV sum_i |V_i . dJU_i - phi_i dJ_i|,
 * where (dJU, dJ) are right-hand sides of eq. semi_U / semi_J at the state (JU, J) (from es_rhs),
 * eta = -rho s, V = eta'(U) the entropy variables, phi = p/T the potential and dV = prod_k dxi_k.  The
 * EC scheme (dissipation = 0) conserves it on periodic data (eq. ECCondition_comp and the telescoping of
 * the EC fluxes), so out_host[0] is round-off of out_host[1]; the ES flux of eq. HOstable only lowers it.
 * Arrays have the state's precision and layout (the mixed form's (hi, lo) planes are read as their sum);
 * the arithmetic is FP64 with a compensated sum in a fixed order, so repeated calls give the same bits.
 * Synchronises the context's stream.  Errors: ES_ERR_ARG for a null pointer. */
int es_entropy_rate(es_ctx* ctx, const void* JU, const void* J, const void* dJU, const void* dJ, double* out_host);

/* Mesh redistribution of Sec. 4 for a step of size dt: monitor (with G) ->
 * filter passes -> Jacobi sweeps from xn -> limiter Delta_gamma -> mesh velocity
 * xdot = Delta_gamma (x^[mu] - xn)/dt.  With a warm-start network registered
 * (es_set_warm_start) the sweeps start, guarded, from its prediction (see
 * es_mesh_solve).  Writes xdot (device) and, if non-null, the sweeps taken and
 * Delta_gamma (host; this synchronises the stream). */
int es_mesh_redistribute(es_ctx* ctx, const void* JU, const void* J, const double* xn,
                         double dt, double* xdot, int* sweeps_host, double* gamma_host);

/* Advance the caller's state (JU, J, x) in place by nsteps full steps
 * (Delta t from eq. cfl or dt_fixed, clipped to t_end; mesh redistribution when
 * moving; three RK stages; x += dt xdot).  On a moving mesh without dt_fixed,
 * eq. cfl's spectral radius holds the step's own mesh velocity (Sec. 4 defines
 * xdot^n = Delta_gamma dx / Delta t_n): Delta t^(0) with the mesh at rest gives
 * xdot, and the step is Delta t_n = min(Delta t^(0), eq. cfl with that xdot), so
 * the mesh moves xdot Delta t_n, within Delta_gamma's bounds.  The time t lives on the device:
 * es_set_time / es_get_time move it.  Steps after t reaches t_end are no-ops.
 * Launches a CUDA graph per step once the first step has been captured. */
int es_steps(es_ctx* ctx, void* JU, void* J, double* x, int nsteps, double t_end);
int es_set_time(es_ctx* ctx, double t);
int es_get_time(es_ctx* ctx, double* t_host, double* last_dt_host);   /* synchronises */

/* One full step (Sec. 4's time step, mesh redistribution and the three SSP-RK3 stages of
 * eq. semi_U / semi_J): es_steps with nsteps = 1.  If t_host or dt_host is non-null it
 * synchronises and writes the time after the step and the step taken (0 once t_end is
 * reached).  Errors as es_steps. */
int es_step(es_ctx* ctx, void* JU, void* J, double* x, double t_end, double* t_host, double* dt_host);

/* End-to-end form for callers holding HOST arrays: copies JU_host, J_host,
 * x_host to context-owned device buffers, runs es_steps, copies them back and
 * synchronises.  Same layouts as the device arrays. */
int es_run_host(es_ctx* ctx, void* JU_host, void* J_host, double* x_host, int nsteps,
                double t_end);

/* Synchronise and return the latched device status (ES_OK or ES_ERR_*);
 * clears it.  es_last_error writes a message (with the first failing node). */
int es_check(es_ctx* ctx);
int es_last_error(es_ctx* ctx, char* buf, int len);

/* Stage-kernel autotuner: times one evaluation of the operator (es_rhs into the
 * context's scratch) for every tile shape on the caller's state and mesh and keeps
 * the fastest for all later launches.  The shapes change only how nodes are
 * grouped into CTAs (how many tiles make a wave on the SMs, how much halo each
 * tile recomputes): in ES_PREC_FP64 every shape gives the same bits, in
 * ES_PREC_MIXED the same values to FP32 rounding.  Writes the
 * chosen shape (1 .. ES_NTILES) and, if ms_host is non-null, the probe times in ms
 * (ES_NTILES of them in 2D; 4 in 3D, the pencil shapes of its direction kernels).  1D contexts have one shape (returns 1).
 * Synchronises. */
int es_autotune(es_ctx* ctx, const void* JU, const void* J, const double* x, int* tile_host, double* ms_host);

/* Device time of the fused stage kernel (Sec. 3 operator + one SSP-RK3 stage, the kernel es_rk_stage runs):
 * `reps` launches of stage `stage` (1..3) with step dt on (JU, J) and the mesh x at rest, back to back on the
 * context's stream between two CUDA events, written to the context's stage buffer; *ms_host = the mean time
 * per launch.  The mixed form's displacement is formed once before the first event.  1D/2D contexts only
 * (ES_ERR_ARG for 3D or reps < 1).  Synchronises the stream. */
int es_time_stage(es_ctx* ctx, const void* JU, const void* J, const double* x, int stage, double dt, int reps,
                  double* ms_host);

/* Self-test of the library's FP64 quotient and reciprocal (the stage kernel divides with
 * them: a Newton-Raphson-refined hardware reciprocal and a Markstein quotient correction):
 * q[i] = a[i] / b[i], r[i] = 1 / b[i] for device arrays of n doubles, on `stream`
 * (asynchronous; ES_ERR_ARG for null arrays or n <= 0, ES_ERR_CUDA if the launch fails).
 * Divisors must be finite, normal and nonzero. */
int es_selftest_division(const double* a, const double* b, double* q, double* r, int64_t n, void* stream);

/* Self-test of the mixed form's arithmetic building blocks, for device arrays of n values (test use):
 * split[2i], split[2i+1] = x[i] as an unevaluated sum hi + lo of two floats taken apart from its bits
 * (|x - hi - lo| < 2^-46 |x| for 2^-103 <= |x| < 2^127, hi the truncation of x); wide[i] = f[i] as a
 * double assembled from its bits (exact, NaN payloads kept); mul[2i..2i+1] and add[2i..2i+1] = the
 * double-float product and sum of (a[2i], a[2i+1]) and (b[2i], b[2i+1]) (the Sec. 3 state arithmetic of
 * the mixed form).  Asynchronous on `stream`; ES_ERR_ARG for a null array or n <= 0, ES_ERR_CUDA if the
 * launch fails. */
int es_selftest_mixed_arith(const double* x, const float* f, const float* a, const float* b, int64_t n,
                            float* split, double* wide, float* mul, float* add, void* stream);

/* Measured arithmetic rates of the current GPU (the roofline denominators of the stage kernels, which the
 * FP64 pipe bounds in the plain form and the FP32 pipe in the mixed and batched forms): a grid of SMs x 8
 * CTAs x 256 threads, each with 8 independent chains of dependent FMAs, timed with CUDA events on `stream`,
 * best of five launches after a warm-up; an FMA counts as two operations.  Writes TFLOP/s to the two host
 * doubles; allocates and frees a small buffer; synchronises `stream`.  About 60 ms.  Errors: ES_ERR_ARG for
 * null outputs, ES_ERR_CUDA. */
int es_selftest_peaks(double* fp64_tflops, double* fp32_tflops, void* stream);

/* Number of kernel launches the library has issued (graph launches count
 * their kernels), for launch accounting. */
int64_t es_launch_count(es_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Learned warm start of the mesh iteration (2D).  The Jacobi iteration of
 * Sec. 4 solves the discretised mesh equation for the new node positions from
 * the monitor omega (after the filter passes); a small network predicts, from
 * omega, the fundamental derivative G and the current mesh, where that
 * iteration ends, and the iteration then starts from the prediction.  The plain
 * iteration always finishes the solve, so the network changes where it starts,
 * never what it converges to; the guard below keeps the plain start whenever the
 * prediction is worse. */

/* Features at the mesh x for the state (JU, J), as float planes [4][n2][n1]
 * (device, caller-owned): ln(omega), G/(1 + |G|), and the displacement of x from
 * the Cartesian mesh (x_00 + i dxi_1, y_00 + j dxi_2) in cells, per direction.
 * omega is the filtered monitor of Sec. 4; G = nu^3 p_nunu|_s / (2 c^2). */
int es_mesh_features(es_ctx* ctx, const void* JU, const void* J, const double* x, float* feat);

/* The Jacobi solve of Sec. 4 alone (no limiter): monitor and filter from (JU, J)
 * on xn, then sweeps until max |x^[nu+1] - x^[nu]| < p->jacobi_eps (if > 0) or
 * p->jacobi_sweeps sweeps.  x_start NULL: from xn.  Otherwise the first sweep
 * runs from both xn and x_start (fixed boundary nodes of x_start must equal xn's),
 * changing the mesh by c0 and c1 (max norm), and x_start is continued if
 * c1 < guard_ratio * c0, else xn.  A ratio above 1 admits a start whose first
 * residual is larger but that lies closer to where the iteration ends; noise at
 * the grid scale, which a plain Jacobi sweep does not damp, gives c1 >> c0.
 * x_out (device [dim][n2][n1], not aliasing xn or x_start; nullable) receives the
 * iterate and disp_out (device float [dim][n2][n1]; nullable, but not both) the
 * displacement (x^[nu] - xn)_k / dxi_k in cells.  If non-null, *sweeps_host =
 * sweeps on the continued path (the guarded first sweep counts once) and
 * *picked_host = 1 if x_start was kept (synchronises). */
int es_mesh_solve(es_ctx* ctx, const void* JU, const void* J, const double* xn, const double* x_start,
                  double guard_ratio, double* x_out, float* disp_out, int* sweeps_host, int* picked_host);

/* x_start = xn + dxi_k out_k (out: device float [2][n2][n1], cells) at the nodes
 * that move; fixed boundary nodes and non-finite outputs keep xn.  The same
 * kernel forms the registered network's warm start. */
int es_mesh_warm_start(es_ctx* ctx, const double* xn, const float* out, double* x_start);

/* Register the warm-start network used by es_mesh_redistribute and es_steps:
 * `layers` 3x3 cross-correlations (zero padding), 4 -> hidden -> ... -> hidden -> 2
 * channels, tanh after all but the last; the output is the displacement in cells,
 * x_start = xn + dxi_k out_k (boundary nodes fixed, non-finite outputs dropped).
 * The layers run as es_nn_conv_forward_bf16 (tensor cores, bf16 layer inputs).
 * w_bf16: device bf16 weights, layer by layer, each [Cout][Cin][3][3]; bias:
 * device float biases, layer by layer.  Both are copied (weights converted to
 * float), so the caller may free or change them afterwards; register again to
 * update.  w_bf16 NULL removes the network.  hidden: 4 or 32; 2 <= layers <= 16.
 * guard_ratio: as in es_mesh_solve. */
int es_set_warm_start(es_ctx* ctx, const uint16_t* w_bf16, const float* bias, int layers, int hidden,
                      double guard_ratio);

/* Cumulative mesh-solve counters of es_mesh_redistribute / es_steps: Jacobi
 * sweeps, solves, and solves that kept the warm start; reset != 0 zeroes them.
 * Synchronises. */
int es_mesh_stats(es_ctx* ctx, int64_t* sweeps_total, int64_t* solves, int64_t* warm_kept, int reset);

/* Network building blocks (training and inference of the warm start), all on
 * device arrays and the given stream.  Activations [B][C][H][W] float, weights
 * [Cout][Cin][3][3] bf16, biases float[Cout]; C in {2, 4, 32}.
 *   forward:  out = act(bias + w (*) in), act = tanh if act_tanh, (*) the 3x3
 *             cross-correlation with zero padding; FP32 accumulation.
 *   backward: given grad_out = dL/d(out) (overwritten by dL/d(pre-activation)
 *             when act_tanh, which needs `out`), writes grad_w = dL/dw and
 *             grad_b = dL/db (summed over the batch, in a fixed order) and, if
 *             grad_in is non-null, grad_in = dL/d(in).
 * workspace: device scratch of at least es_nn_workspace_bytes(B, Cin, Cout, H, W)
 * bytes (forward needs only Cout*Cin*9 floats).  Returns ES_ERR_ARG for bad
 * shapes, null pointers or aliasing outputs. */
size_t es_nn_workspace_bytes(int B, int Cin, int Cout, int H, int W);
/* Forward layer on the tensor cores (the warm start's inference path): the same
 * correlation with the layer input rounded to bf16 (round to nearest even), bf16
 * weights, products accumulated in FP32 (mma m16n8k16), bias and tanh in FP32. */
int es_nn_conv_forward_bf16(const float* in, const uint16_t* w, const float* bias, float* out, int B, int Cin,
                            int Cout, int H, int W, int act_tanh, void* stream);
int es_nn_conv_forward(const float* in, const uint16_t* w, const float* bias, float* out, int B, int Cin, int Cout,
                       int H, int W, int act_tanh, void* workspace, size_t workspace_bytes, void* stream);
int es_nn_conv_backward(const float* in, const uint16_t* w, const float* out, float* grad_out, float* grad_in,
                        float* grad_w, float* grad_b, int B, int Cin, int Cout, int H, int W, int act_tanh,
                        void* workspace, size_t workspace_bytes, void* stream);
/* dst = src rounded to the nearest bf16 (ties to even), n elements. */
int es_nn_to_bf16(const float* src, uint16_t* dst, int64_t n, void* stream);
/* *loss += mean((pred - target)^2) over n elements; grad = 2 (pred - target)/n. */
int es_nn_mse(const float* pred, const float* target, float* grad, float* loss, int64_t n, void* stream);
/* One Adam step (Kingma & Ba 2015, bias-corrected, step >= 1) on FP32 master
 * weights with moments m, v; if w_bf16 is non-null it receives the master rounded
 * to nearest bf16. */
int es_nn_adam(float* master, uint16_t* w_bf16, const float* grad, float* m, float* v, int n, float lr, float beta1,
               float beta2, float eps, int step, void* stream);

/* ---------------------------------------------------------------------------
 * Batched form: many independent 1D problems (shock tubes on [0, 1], outflow
 * boundaries, uniform initial mesh x_i = i/(L_p - 1)) advanced together by one
 * persistent kernel replayed from a CUDA graph.  Each CTA takes a whole problem
 * from a work queue (longest first) and runs its full steps -- its own CFL time
 * step (eq. cfl), its own mesh redistribution (Sec. 4) and the three SSP-RK3
 * stages of the fused operator -- with no waits on other CTAs.  Arithmetic is the
 * mixed form (FP32 pipe, double-float state); the mesh is kept as an FP32
 * displacement from the uniform mesh.  Packed layout: node i of problem p is
 * element off_p + i, off_p = sum of the earlier lengths; ntot = sum of lengths. */
typedef struct es_batch es_batch;

/* p: gas, WENO, CFL and mesh parameters; p->dim must be 1 and p->precision
 * ES_PREC_MIXED (n1, n2, dxi, period and bc are ignored).  lengths_host: nodes of
 * each problem (>= 8).  Allocates the packed state and scratch. */
int es_batch_create(es_batch** b, const es_params* p, int nprob, const int* lengths_host, void* stream);
void es_batch_destroy(es_batch* b);
int64_t es_batch_nodes(es_batch* b);
/* Initial primitive state of every node (device arrays of ntot doubles). */
int es_batch_set_prim(es_batch* b, const double* rho, const double* v, const double* p);
/* State of every problem from conservative values, as es_batch_get returns them (device arrays): JU [3][ntot],
 * J [ntot] and x [ntot] (node coordinates, x_0 = 0 and x_{L-1} = 1 for outflow ends), and t [nprob] the time of
 * each problem.  JU and J are split into the form's (hi, lo) float planes, x into the FP32 displacement from
 * the uniform mesh; the mesh velocity restarts at zero (each step recomputes it).  Restarts a batch, or sets
 * each problem to a given step of a reference run. */
int es_batch_set_state(es_batch* b, const double* JU, const double* J, const double* x, const double* t);
/* Advance every problem by nsteps full steps (each clipped to t_end). */
int es_batch_steps(es_batch* b, int nsteps, double t_end);
/* Autotuner of the CTA shape: runs one step of every shape the library has
 * (128, 256 or 512 threads per CTA, stage chunks of threads - 2 nodes; the grid
 * is SMs x resident CTAs of that shape) from the current state, restores the
 * state, and keeps the fastest for the following es_batch_steps.  Writes the
 * chosen threads per CTA and, if ms_host is non-null, the three probe times
 * (ms).  Needs a temporary copy of the state (26 floats per node).  Synchronises. */
int es_batch_autotune(es_batch* b, int* bt_host, double* ms_host);
/* State as doubles: JU [3][ntot], J [ntot], x [ntot]; t [nprob] (nullable).  Device arrays. */
int es_batch_get(es_batch* b, double* JU, double* J, double* x, double* t);
int es_batch_check(es_batch* b);                      /* synchronises; latched device status */
int es_batch_last_error(es_batch* b, char* buf, int len);

/* ---------------------------------------------------------------------------
 * Allocation-free SSP-RK3 step.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc (a host application
 * that owns and budgets all device memory itself, code running while a memory
 * pool is torn down or rebuilt, a process that must not allocate after its
 * start-up).  It needs no es_ctx.
 *
 * Advances (JU, J) in place by one SSP-RK3 step of size dt of the FP64
 * operator (the same three fused stage launches as es_rk_stage), on the mesh x
 * moving with velocity xdot (nullable: fixed mesh); x itself is not updated.
 * p must have precision ES_PREC_FP64; the time-step, mesh and graph fields of
 * p are ignored.  All arrays are caller-owned device arrays as above.
 *
 * Scratch: the two intermediate stage states and the status word live in a
 * __device__ array compiled into the library (about 5 MB, held on every GPU
 * that loads the library until the process exits).  Meshes with more than
 * ES_STATIC_MAX_NODES nodes are rejected with ES_ERR_ARG.  The call allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 *
 * The first call on a device does that device's set-up, with it current: it
 * looks up the scratch array's device address and sets the stage kernel's
 * shared-memory attribute.  Under CUDA's lazy module loading (the default) that
 * is also when the driver loads the library's modules, and with them reserves
 * the scratch array, so the first call on each device can itself take device
 * memory.  Make it during start-up, before the program stops allocating and
 * before any stream capture (or set CUDA_MODULE_LOADING=EAGER so the modules
 * and the array are loaded when the context is created).  es_params.tile picks
 * the 2D stage tile as in es_create (0: the default shape).  Every call then clears the
 * status word, launches on `stream` and synchronises it to read the status
 * back: the return value is ES_OK, ES_ERR_ARG, ES_ERR_CUDA, or a device status
 * such as ES_ERR_INADMISSIBLE.  All calls share the one scratch array and it
 * keeps the last call's contents, so calls that overlap on the GPU (from two
 * streams or two host threads) race on it and must be serialised by the
 * caller. */
#define ES_STATIC_MAX_NODES 65536
int es_rk3_step_static(const es_params* p, double dt, double* JU, double* J, const double* x,
                       const double* xdot, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ES_VDW_H */
