/*
 * gs.h -- C ABI of the B300 explicit time-stepping library (libgs_b300.so).
 *
 * The library integrates du/dt = F(t,u), u(0) = u0 (paper, Introduction) with
 * the explicit steppers of Table 1 that are in scope here: fixed-step
 * explicit Euler, Runge-Kutta 4 and Dormand-Prince 5, error-controlled
 * Dormand-Prince 5(4), and Adams-Bashforth 4.  F is either the 3D Gray-Scott
 * reaction-diffusion system (Eq. 2, with the v-equation as in the System
 * functor of Listing 2) on a periodic grid with the 7-point central
 * Laplacian, or a pointwise ODE applied to every element of a vector.
 *
 * Conventions shared by every entry point
 *   - Device arrays are owned by the caller (e.g. PyTorch tensors); the
 *     library never frees them.  Pointers named *_dev / state pointers are
 *     device pointers; pointers named *_host are host pointers.
 *   - Gray-Scott state: two arrays u and v (structure of arrays), each of
 *     nx*ny*nz elements of the context's precision, cell (x,y,z) at index
 *     x + nx*(y + ny*z) (x fastest), 16-byte aligned.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; calls that return host-side results (t, dt, step
 *     counts, norms) synchronise that stream before returning.
 *   - Every call returns a gs_status and never aborts.  On GS_ERR_CUDA the
 *     CUDA error text is available from gs_last_error(ctx) (or
 *     gs_last_global_error() for context-free calls).
 *   - Time t and step sizes are FP64 on the host and on the device in every
 *     precision; only the bulk stencil / stage arithmetic follows the
 *     context precision.
 *   - The library has no CPU fallback: without a usable CUDA device every
 *     compute call fails with GS_ERR_CUDA.
 */
#ifndef GS_B300_H
#define GS_B300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID = 1,        /* bad argument: null pointer, size, enum, unbound state */
    GS_ERR_CUDA = 2,           /* a CUDA runtime call failed (see gs_last_error) */
    GS_ERR_NOMEM = 3,          /* device or pinned host allocation failed */
    GS_ERR_STEP_UNDERFLOW = 4, /* adaptive control: 500 consecutive rejections, or t + dt == t */
    GS_ERR_MAX_STEPS = 5,      /* adaptive control: attempt limit reached before t_end */
    GS_ERR_NONFINITE = 6       /* adaptive control: error norm is NaN or infinite */
} gs_status;

typedef enum { GS_FP64 = 0, GS_FP32 = 1 } gs_precision;

/* Steppers of Table 1 available through gs_step / ode_integrate_const. */
typedef enum {
    GS_RK4 = 0,    /* classical Runge-Kutta 4, fixed step */
    GS_DOPRI5 = 1, /* Dormand-Prince 5 (its 5th-order solution), fixed step */
    GS_AB4 = 2,    /* Adams-Bashforth 4; the first 3 steps of each call by RK4 */
    GS_EULER = 3,  /* explicit Euler */
    GS_CK54 = 4,    /* Cash-Karp 5(4) (its 5th-order solution), fixed step */
    GS_RKF78 = 5,   /* Fehlberg 7(8) (its 8th-order solution, 13 stages), fixed step */
    GS_MIDPOINT = 6 /* modified midpoint, two substeps of dt/2 (order 2), fixed step */
} gs_method;

/* Gray-Scott problem (Eq. 2): periodic box [0,Lx)x[0,Ly)x[0,Lz), nx*ny*nz
 * cells, spacing h_d = L_d / n_d, diffusivities Du, Dv, feed rate F and kill
 * rate k:  du/dt = Du Lap(u) - u v^2 + F (1 - u),
 *          dv/dt = Dv Lap(v) + u v^2 - (F + k) v.
 * prec is a gs_precision. */
typedef struct {
    int nx, ny, nz;
    double Lx, Ly, Lz;
    double Du, Dv, F, k;
    int prec;
} gs_params;

typedef struct gs_ctx gs_ctx; /* opaque; owns the stage scratch (the state type's
                                 temporaries of the section "Architecture and
                                 nomenclature of Boost Odeint") */

/* Creates a context for one Gray-Scott problem on the current device.  Stage
 * scratch (8 fields x 2 components) and a small control block are allocated
 * here (the Algebra's resize, section "The distributed OpenFPM state type and
 * algebra").  Requires 1 <= n_d <= 65535, L_d > 0.
 * stream: where all work of this context is enqueued.
 * Errors: INVALID (p/out NULL, bad sizes), NOMEM, CUDA. */
gs_status gs_create(const gs_params* p, void* stream, gs_ctx** out);

/* Frees the context's scratch and graphs (not the bound state).  NULL is a no-op. */
gs_status gs_destroy(gs_ctx* ctx);

/* Binds the caller-owned device arrays u and v (nx*ny*nz elements each, of
 * the context precision).  All integrators update them in place (section
 * "Reuse potential": the state is updated in-place).  INVALID if NULL or not
 * 16-byte aligned. */
gs_status gs_bind_state(gs_ctx* ctx, void* u_dev, void* v_dev);

/* Copies host arrays into the bound state (stream-ordered; returns once the
 * copies are enqueued; host buffers must stay valid until the stream passes
 * them -- pinned memory gives asynchronous copies). */
gs_status gs_upload_state(gs_ctx* ctx, const void* u_host, const void* v_host);

/* Copies the bound state to host arrays and synchronises the stream. */
gs_status gs_download_state(gs_ctx* ctx, void* u_host, void* v_host);

/* One evaluation of the System F(t, (u,v)) (Listing 2):
 * (fu, fv) = F(t, (u, v)).  All four are device arrays of nx*ny*nz elements,
 * 16-byte aligned (else INVALID); outputs must not alias inputs.  Enqueued
 * on the context stream. */
gs_status gs_rhs(gs_ctx* ctx, double t, const void* u_dev, const void* v_dev, void* fu_dev,
                 void* fv_dev);

/* integrate_const / do_step (Listing 3): nsteps fixed steps of size dt from
 * *t on the bound state.  Step m is taken at time *t + m*dt; on return
 * *t = *t + nsteps*dt.  nsteps = 0 is a no-op.  GS_CK54, GS_RKF78 and
 * GS_MIDPOINT run on the tableau path (see gs_set_laplacian; Fehlberg's
 * stage fields k8..k13 and one more stage-input buffer are allocated at the
 * first call that needs them, 7 fields x 2 components).  Synchronises the
 * stream. */
gs_status gs_step(gs_ctx* ctx, gs_method method, double* t, double dt, long nsteps);

/* integrate_adaptive (section "Architecture and nomenclature of Boost
 * Odeint"): error-controlled Dormand-Prince 5(4) on the bound state from *t
 * towards t_end with initial step *dt and tolerances atol, rtol.
 * Error norm: E = max over cells and both components of
 *   |err_i| / (atol + rtol (|u_i| + dt |k1_i|)),   err = dt sum_j (b_j - bhat_j) k_j.
 * Step-size controller (paper silent; this library's reading):
 *   E > 1 reject, dt *= max(0.9 E^(-1/3), 0.2);
 *   E < 0.5 accept, dt *= 0.9 max(E, 5^-5)^(-1/5);  otherwise accept, dt kept.
 * The last step is clipped to land exactly on t_end.  Integration stops at
 * t_end or after max_accepted accepted steps (max_accepted < 0: no limit;
 * t_end may be +inf then).  On return *t, *dt (the next proposed step),
 * *n_accepted, *n_rejected are set (the latter two may be NULL).
 * Statuses: STEP_UNDERFLOW, NONFINITE, MAX_STEPS (more than 10^7 attempts).
 * In FP32 contexts the per-cell scaled errors are formed in FP32 from the
 * FP32 stage values; the max-reduction, controller, dt and t are FP64.
 * Synchronises the stream. */
gs_status gs_integrate_adaptive(gs_ctx* ctx, double atol, double rtol, double* t, double t_end,
                                double* dt, long max_accepted, long* n_accepted,
                                long* n_rejected);

/* integrate_adaptive with another error stepper of Table 1: pair =
 * GS_DOPRI5 (the same as gs_integrate_adaptive), GS_CK54 (Cash-Karp 5(4),
 * orders p = 5, q = 4) or GS_RKF78 (Fehlberg 7(8): the order-8 solution
 * propagated, the order-7 one embedded, p = 8, q = 7).  Same norm,
 * clipping, limits and results as gs_integrate_adaptive; the controller
 * takes the pair's orders: E > 1 reject, dt *= max(0.9 E^(-1/(q-1)), 0.2);
 * E < 0.5 accept, dt *= 0.9 max(E, 5^-p)^(-1/p); otherwise accept, dt
 * kept.  Cash-Karp and Fehlberg run on the tableau path described at
 * gs_set_laplacian (one tiled stage kernel per stage, the controller on
 * the host), with either Laplacian.  INVALID: any other pair. */
gs_status gs_integrate_adaptive_pair(gs_ctx* ctx, gs_method pair, double atol, double rtol, double* t,
                                     double t_end, double* dt, long max_accepted, long* n_accepted,
                                     long* n_rejected);

/* Observer (the functor Odeint calls before each time step, e.g. to write
 * output; section "Architecture and nomenclature of Boost Odeint"):
 * fn(t, u, v, user) runs on the calling host thread with u, v the device
 * pointers of the state bound to ctx, after ctx's stream has drained; it
 * may read them (on any stream) but must not write them.  With an observer
 * set, gs_step calls it at t0, t0 + dt, ..., t0 + nsteps dt (before each
 * step and once after the last), and gs_integrate_adaptive at the start
 * time and after every accepted step.  A nonzero return stops the call
 * before its next step: it returns GS_OK with *t (and *dt, *n_accepted,
 * *n_rejected) describing the steps taken.  The observed run launches
 * each step on its own and synchronises after it, with the device control
 * block carried from step to step, so its steps, its states and its
 * results are those of the same call without an observer.  fn = NULL
 * removes the observer; the library never frees `user`.  The observer is
 * not called by the batched integrator (gsb_*). */
typedef int (*gs_observer)(double t, void* u, void* v, void* user);
gs_status gs_set_observer(gs_ctx* ctx, gs_observer fn, void* user);

/* Enables (capacity > 0) or disables (0) recording of the accepted step
 * sizes of later gs_integrate_adaptive calls into a device buffer of
 * `capacity` doubles. */
gs_status gs_set_step_log(gs_ctx* ctx, long capacity);

/* Copies up to `capacity` recorded step sizes to dts_host; *count receives
 * the number recorded by the last call (may exceed capacity). Synchronises. */
gs_status gs_get_step_log(gs_ctx* ctx, double* dts_host, long capacity, long* count);


/* Project autotuner: for each kernel of a Dormand-Prince attempt (k1 and
 * stages 2..7) times every candidate kernel form allowed by the variant
 * setting and every candidate tile (ty, zc), each launched alone from the
 * bound state (outputs go to the context's scratch; the bound state is not
 * modified), and keeps the fastest per kernel.  RK4, Euler, Adams-Bashforth
 * and gs_rhs then use stage 2's configuration.  *ty, *zc: that
 * configuration's tile; *best_ms: the sum of the best kernel times.  ty, zc
 * and best_ms may be NULL. */
gs_status gs_autotune(gs_ctx* ctx, int* ty, int* zc, double* best_ms);

/* Laplacian of the Gray-Scott right-hand side.  GS_LAP_7POINT (default):
 * the 7-point central stencil of the stage kernels.  GS_LAP_DCPSE: the
 * DC-PSE operator the paper's Gray-Scott benchmark uses (discretization-
 * corrected particle strength exchange, cited, not specified, by the paper).
 * This library's reading: Gaussian kernel, eps = h_d per axis, convergence
 * order 2 (moment conditions on every monomial of degree 1..3), support all
 * grid points within rc_over_h spacings (3.1: 122 neighbours); on the
 * regular grid the operator is one stencil L f_p = sum_q w_q (f_{p+o_q} -
 * f_p), whose weights gs_set_laplacian computes once (Cholesky of the
 * moment system; the solved weights are even in the offset and are stored
 * exactly so, each pair {o, -o} taking the mean of its two values).  With
 * GS_LAP_DCPSE, gs_rhs, gs_step (GS_EULER, GS_RK4, GS_DOPRI5, GS_CK54,
 * GS_RKF78; GS_AB4 -> INVALID), gs_integrate_adaptive and
 * gs_integrate_adaptive_pair run the tableau path: one tiled stage kernel
 * per stage (8 x 8 x 8 or 8 x 8 x 4 cells + a halo of 3 in shared memory),
 * each stage also forming the next stage's input at its own cells and the
 * last one the new state (and the attempt's error maximum), the adaptive
 * controller on the host with the formulas and limits of the graph path;
 * synchronous.  The FP64 kernel sums the stencil over the offset pairs,
 * sum_k w_k (f_{p+o_k} + f_{p-o_k}) - (sum_q w_q) f_p.  Cash-Karp and
 * Fehlberg take the same path with the 7-point Laplacian too (as the
 * stencil of the six neighbours, halo 1).
 * INVALID: unknown kind, rc_over_h outside [2, 4), a singular moment
 * system.  gs_get_dcpse_stencil: the offsets (3 ints each, in spacings)
 * and weights in use; capacity = 0 returns the count only.
 */
typedef enum { GS_LAP_7POINT = 0, GS_LAP_DCPSE = 1 } gs_laplacian;
gs_status gs_set_laplacian(gs_ctx* ctx, gs_laplacian kind, double rc_over_h);
gs_status gs_get_dcpse_stencil(const gs_ctx* ctx, int* count, int* offsets, double* weights, int capacity);

/* Text of the last CUDA error seen by ctx ("" if none). */
const char* gs_last_error(const gs_ctx* ctx);
/* Text of the last CUDA error seen by a context-free entry point. */
const char* gs_last_global_error(void);

/* ------------------------------------------------------------------------ */
/* Batched ensembles: many independent Gray-Scott problems of uneven sizes    */
/* and parameters, each with its own adaptive step (the error-controlled    */
/* integrate_adaptive of section "Architecture and nomenclature of Boost    */
/* Odeint", applied per instance)                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz; /* grid of this instance, each 1..65535 */
    double F, k;    /* feed and kill rates of this instance */
} gsb_instance;

typedef struct gsb_ctx gsb_ctx; /* opaque; owns the stage scratch of all instances */

/* Creates an ensemble of `count` (1..65536) instances, each on the periodic
 * box [0,L)^3 with spacing L/n_d per axis, shared diffusivities Du, Dv and
 * precision prec.  The instances' states are concatenated in two arrays
 * (u, v) at the element offsets reported by gsb_layout (each 16-byte
 * aligned, cell (x,y,z) of instance i at offset_i + x + nx_i (y + ny_i z)).
 * Errors: INVALID, NOMEM, CUDA. */
gs_status gsb_create(int count, const gsb_instance* inst, double L, double Du, double Dv, int prec,
                     void* stream, gsb_ctx** out);
gs_status gsb_destroy(gsb_ctx* ctx);

/* offsets[i] = element offset of instance i, offsets[count] = total length
 * of each state array.  offsets: host array of count + 1. */
gs_status gsb_layout(const gsb_ctx* ctx, long long* offsets);

/* Binds the caller-owned concatenated state arrays (total length each, of
 * the ensemble precision, 16-byte aligned); updated in place. */
gs_status gsb_bind_state(gsb_ctx* ctx, void* u_dev, void* v_dev);

/* Error-controlled Dormand-Prince 5(4) for every instance from t[i] towards
 * t_end with its own step size: same norm, controller and clipping as
 * gs_integrate_adaptive, decided per instance.  Each Dormand-Prince stage of
 * all instances is one persistent kernel launch (CTAs take segments of any
 * running instance from an atomic counter); the stage loop is one CUDA graph
 * (WHILE any instance is running).  t, dt: host arrays of count, in/out.
 * n_acc, n_rej, status: optional host arrays of count.  Returns GS_OK if
 * every instance ended OK, else the first failing instance's status (the
 * others are integrated regardless).  Synchronises the stream. */
gs_status gsb_integrate_adaptive(gsb_ctx* ctx, double atol, double rtol, double* t, double t_end,
                                 double* dt, long max_accepted, long* n_acc, long* n_rej,
                                 int* status);


/* Project autotuner for the batched kernels: times one Dormand-Prince attempt
 * of the bound ensemble for each candidate segment shape and keeps the
 * fastest (the bound state is not modified). */
gs_status gsb_autotune(gsb_ctx* ctx, int* ty, int* zc, double* best_ms);
/* Tile choice by timing the caller's integration itself: each candidate
 * (the single-stage kernels at 7 tile shapes; the stage pairs, stages 2+3,
 * 4+5 and 6+7 each one step, at 6 tile shapes for the instances run with
 * one cell per lane; the instances whose rows allow 2 or 4 cells per lane
 * run so at tile height 7 in their own launches, as gsb_set_pair_lanes in
 * the internal header describes)
 * runs gsb_integrate_adaptive(atol, rtol, t0 -> t_end, dt0 for every
 * instance) twice (the first run builds its graph) from the bound state,
 * which is saved (a temporary copy of the state, allocated and freed here)
 * and restored after every run and at the end; the fastest second run
 * wins.  Unlike gsb_autotune's dense timing round, a real run of an uneven
 * ensemble has instances finishing at different times.  Grouping is left as
 * set.  Synchronises; INVALID for t0 >= t_end, dt0 <= 0 or bad tolerances. */
gs_status gsb_autotune_run(gsb_ctx* ctx, double atol, double rtol, double t0, double t_end, double dt0, int* ty_out,
                           int* zc_out, double* best_ms);

/* Records the accepted step sizes of every instance in later
 * gsb_integrate_adaptive calls (capacity per instance; 0 disables; device
 * memory of count x capacity doubles allocated here).  gsb_get_step_log
 * copies them to dts_host (count x capacity doubles, instance-major; the
 * entries past an instance's count are untouched) and its accepted counts
 * to counts (host array of count; a count may exceed capacity, only the
 * first capacity sizes are kept).  capacity <= the logging capacity;
 * synchronises.  With the sizes a run can be replayed step for step. */
gs_status gsb_set_step_log(gsb_ctx* ctx, long capacity);
gs_status gsb_get_step_log(gsb_ctx* ctx, double* dts_host, long capacity, long* counts);

const char* gsb_last_error(const gsb_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Learned surrogate of the Gray-Scott integrator (the paper has no learned  */
/* part: a BF16 3D convolutional network trained on the integrator's own    */
/* trajectories, with the RK4 integrator as judge and fallback)              */
/* ------------------------------------------------------------------------ */
/* Network: x0 = ((u - mu_u)/sd_u, (v - mu_v)/sd_v); a_l = relu(conv_l(a_{l-1}))
 * for l = 1..3 (2 -> 32 -> 32 -> 32 channels); y = conv_4(a_3) (32 -> 2);
 * prediction of the state 16 RK4 steps (dt = 0.1) ahead = (u, v) + s * y.
 * conv_l: 3x3x3 periodic convolution + bias, BF16 weights and activations
 * (channels-last), FP32 accumulation on the tensor cores.  Parameters: one
 * FP32 vector, per layer W[27][cin][cout] (tap = (dz+1)*9 + (dy+1)*3 +
 * (dx+1)) then b[cout]. */
typedef struct sur_ctx sur_ctx;
/* Failure of the tensor-core kernels: every wait they make for their MMAs
 * is bounded; a launch that gives up frees its tensor memory, returns, and
 * marks its context failed (its outputs are invalid).  From then on every
 * call on the context returns GS_ERR_CUDA (sur_last_error says why), and a
 * synchronising call (sur_train_step with loss, sur_advance, sur_get_params,
 * sur_get_grad) reports its own launches' failure before it returns, so no
 * result computed by a failed launch is reported as a success.  The calls
 * that only enqueue work (sur_forward, sur_train_step without loss) report
 * it at the next call.  The layer primitives (sur_conv3d,
 * sur_conv3d_wgrad) share one process-wide failure mark in the same way. */

/* Length of the parameter vector (58,850). */
long sur_param_count(void);

/* Context for one grid (nx % 16 == 0, ny % 8 == 0, nz % 2 == 0): parameters,
 * Adam moments, activations and gradients (about 280 B per cell). */
gs_status sur_create(int nx, int ny, int nz, void* stream, sur_ctx** out);
gs_status sur_destroy(sur_ctx* ctx);

/* Host copies of the FP32 parameters (set resets the Adam moments). */
gs_status sur_set_params(sur_ctx* ctx, const float* params_host);
gs_status sur_get_params(sur_ctx* ctx, float* params_host);
/* Gradient of the last sur_train_step's loss w.r.t. the parameters. */
gs_status sur_get_grad(sur_ctx* ctx, float* grad_host);

/* Per-channel input mean mu and deviation sd, increment scale s (host
 * arrays of 2 doubles: u, v). */
gs_status sur_set_normalization(sur_ctx* ctx, const double* mean, const double* sd, const double* scale);

/* Prediction (u_out, v_out) of the state 16 RK4 steps ahead of (u, v).
 * FP32 device arrays of nx*ny*nz cells (x fastest); outputs must not alias
 * inputs.  Enqueued on the context stream. */
gs_status sur_forward(sur_ctx* ctx, const float* u, const float* v, float* u_out, float* v_out);

/* One Adam step (beta = 0.9, 0.999, eps = 1e-8, learning rate lr) on the
 * mean squared error of the normalised increment (u_tgt - u)/s_u,
 * (v_tgt - v)/s_v over all cells; *loss (may be NULL) = the loss before the
 * step.  Forward, input-gradient and weight-gradient convolutions all run on
 * the BF16 tensor-core kernels.  Synchronises if loss != NULL. */
gs_status sur_train_step(sur_ctx* ctx, const float* u, const float* v, const float* u_tgt, const float* v_tgt,
                         double lr, double* loss);

/* Advances (u, v) by 1.6 time units.  integ: a GS_FP32 context of the same
 * grid bound to u, v (RK4, dt = 0.1, 16 steps).  judge = 0: the surrogate's
 * prediction replaces (u, v) -- unless the last judged call failed, in which
 * case the integrator runs (plain RK4 fallback, *fell_back = 1).  judge = 1:
 * both run, (u, v) receive the integrator's result, *rel_err = relative L2
 * distance of the prediction from it, and the context falls back to RK4 for
 * later unjudged calls while *rel_err > threshold.  Synchronises. */
gs_status sur_advance(sur_ctx* ctx, gs_ctx* integ, float* u, float* v, int judge, double threshold,
                      double* rel_err, int* fell_back);

const char* sur_last_error(const sur_ctx* ctx);

/* Layer-level primitives.  Channel counts are padded to 8 or 32 in memory
 * (BF16, channels-last, 16-byte cells); D % 2 == 0, H % 8 == 0, W % 16 == 0. */
/* Packed tensor-core weight operand of a layer with real channels (cin,
 * cout) from W[27][cin][cout] (FP32 device array): dgrad = 0 for the
 * forward convolution, 1 for its input-gradient convolution (taps mirrored,
 * channel roles swapped).  packed: device buffer of
 * sur_packed_bytes(pad(cin), pad(cout)) (forward) or sur_packed_bytes(
 * pad(cout), pad(cin)) (input gradient) bytes. */
size_t sur_packed_bytes(int cin_pad, int cout_pad);
gs_status sur_pack_weights(int cin, int cout, const float* w_dev, int dgrad, void* packed_dev, void* stream);
/* out = epi(conv(x, packed)); epi 0: + bias, ReLU, BF16 [cells][cout_pad];
 * 1: + bias, FP32 [cells][out_ch]; 2: times (mask > 0) (mask BF16
 * [cells][cout_pad]), BF16; 3: FP32 [cells][cout_pad] (+ bias if given). */
gs_status sur_conv3d(int D, int H, int W, int cin_pad, int cout_pad, const void* x, const void* packed,
                     const float* bias, int epi, const void* mask, void* out, int out_ch, void* stream);
/* dw[27][cin][cout] (FP32) = sum over cells p of x[p + off(tap)][i] dy[p][o]
 * (the weight gradient); workspace of sur_wgrad_workspace_bytes bytes. */
size_t sur_wgrad_workspace_bytes(int cin_pad, int cout_pad);
gs_status sur_conv3d_wgrad(int D, int H, int W, int cin_pad, int cout_pad, const void* x, const void* dy, int cin,
                           int cout, float* dw, void* workspace, size_t ws_bytes, void* stream);
/* sum_sumsq_dev[0] += sum x, [1] += sum x^2 (FP64, device). */
gs_status sur_moments(long n, const float* x, double* sum_sumsq_dev, void* stream);

/* ------------------------------------------------------------------------ */
/* Stage algebra (section "The distributed OpenFPM state type and algebra":  */
/* for_each operations over up to 15 states)                                 */
/* ------------------------------------------------------------------------ */

/* y[i] = sum_{j<nterms} coef[j] * x_j[i] for i < n.  coef: host array of
 * nterms doubles (cast to the precision of the data).  x: host array of
 * nterms device pointers (each n elements of precision prec, 16-byte
 * aligned); y may alias one of them.  1 <= nterms <= 15, n >= 0.  Enqueued
 * on stream. */
gs_status ode_axpy_stage(long n, gs_precision prec, int nterms, const double* coef,
                         const void* const* x, void* y, void* stream);

/* ------------------------------------------------------------------------ */
/* Pointwise ODE ensembles: dx_i/dt = f(x_i) on n independent FP64 elements */
/* (autonomous forms of the benchmark families of "Accuracy Benchmarks")    */
/* ------------------------------------------------------------------------ */
typedef enum {
    ODE_EXP_DECAY = 0,    /* f(x) = -x,        x(t) = x0 e^-t */
    ODE_LOGISTIC = 1,     /* f(x) = x (1 - x), x(t) = x0 / (x0 + (1 - x0) e^-t) */
    ODE_PAPER_EXP = 2,    /* Eq. 1a: f(t) = c_i e^t (c_i = x y of element i), u = c_i e^t */
    ODE_PAPER_SIGMOID = 3 /* Eq. 1b: f(t) = s (1 - s), s = 1 / (1 + e^-t), u = s(t) */
} ode_rhs;
/* (ODE_PAPER_EXP and ODE_PAPER_SIGMOID: ode_integrate_tableau,
 * ode_integrate_ab_steps and ode_integrate_adaptive_each only.) */

/* Explicit Runge-Kutta tableaux of Table 1 for the pointwise ensembles. */
typedef enum {
    ODE_TAB_EULER = 0,
    ODE_TAB_RK4 = 1,
    ODE_TAB_DOPRI5 = 2, /* Dormand-Prince 5(4), order 5 propagated */
    ODE_TAB_CK54 = 3,   /* Cash-Karp 5(4), order 5 propagated */
    ODE_TAB_RKF78 = 4,   /* Fehlberg 7(8), 13 stages, order 8 propagated */
    ODE_TAB_MIDPOINT = 5 /* modified midpoint: z1 = x + h f(x), z2 = x + 2h f(z1),
                            x' = (z1 + z2 + h f(z2)) / 2, h = dt / 2 (order 2) */
} ode_tableau;

/* Workspace bytes needed by ode_integrate_adaptive for n elements. */
size_t ode_workspace_size(long n);

/* Error-controlled Dormand-Prince 5(4) on x (n FP64 device values) with ONE
 * global step size (a single state vector with a global norm, section
 * "Architecture and nomenclature of Boost Odeint"); same norm, controller
 * and clipping as gs_integrate_adaptive.  workspace: device buffer of at
 * least ode_workspace_size(n) bytes, 256-byte aligned, owned by the caller.
 * dt_log: optional device array (may be NULL) receiving the accepted step
 * sizes, up to log_cap entries.  max_steps bounds accepted steps (< 0: none).
 * Synchronises the stream. */
gs_status ode_integrate_adaptive(ode_rhs rhs, long n, double* x_dev, double* t, double t_end,
                                 double* dt, double atol, double rtol, long max_steps,
                                 long* n_acc, long* n_rej, void* workspace,
                                 size_t workspace_bytes, double* dt_log, long log_cap,
                                 void* stream);

/* Allocation-free form of ode_integrate_adaptive (the paper has no
 * counterpart; it exists for callers that cannot allocate GPU memory when
 * they integrate: a host application that owns every device allocation
 * through its own pool, a real-time loop where cudaMalloc's implicit device
 * synchronisation and latency are not allowed, or a plugin that may only use
 * memory it was handed).  Same method, norm, controller, arguments and
 * results as ode_integrate_adaptive, without the workspace and step log: its
 * scratch (control block + one second state buffer) is a static device array
 * of 256 B + 8 MiB compiled into the library, which every GPU that loads the
 * library holds until the process exits.
 *   - n must be <= 1048576 (2^20) elements, else GS_ERR_INVALID with the
 *     reason in gs_last_global_error().
 *   - Calls no cudaMalloc/cudaFree and allocates no host or device memory;
 *     the attempts are driven by a host loop (one stream synchronisation per
 *     16 attempts) instead of a graph.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call on a device shares the one array and rewrites its control
 *     block at the start; calls that overlap on the GPU (other streams, other
 *     host threads) race on it and must be serialised by the caller.
 * Synchronises the stream. */
gs_status ode_integrate_adaptive_noalloc(ode_rhs rhs, long n, double* x_dev, double* t,
                                         double t_end, double* dt, double atol, double rtol,
                                         long max_steps, long* n_acc, long* n_rej, void* stream);

/* Adams-Bashforth 4 (Table 1) for nsteps steps of size dt from t0; the first
 * three steps by RK4.  All steps of an element run in registers in one
 * kernel (no global synchronisation is needed between fixed steps).
 * Enqueued on stream. */
gs_status ode_integrate_ab4(ode_rhs rhs, long n, double* x_dev, double t0, double dt, long nsteps,
                            void* stream);

/* Fixed-step Euler / RK4 / Dopri5 (Table 1), nsteps steps of dt, in
 * registers, one kernel.  Enqueued on stream. */
gs_status ode_integrate_const(ode_rhs rhs, gs_method method, long n, double* x_dev, double t0,
                              double dt, long nsteps, void* stream);

/* Fixed-step explicit Runge-Kutta with tableau `method` (Table 1) on n
 * independent FP64 elements x (device), t_m = t0 + m dt, nsteps steps; all
 * stages and steps of an element in registers, one kernel.  coef: device
 * array of n coefficients c_i, required for ODE_PAPER_EXP, else ignored
 * (may be NULL).  INVALID: unknown kind or method, n < 0, nsteps < 0,
 * non-finite t0 or dt, coef missing for ODE_PAPER_EXP.  Enqueued on stream.
 * ODE_PAPER_EXP / ODE_PAPER_SIGMOID depend on the element only through a
 * factor of t shared by all elements, so the call first tabulates that
 * factor at every stage time (a stream-ordered temporary allocation of 8
 * bytes per step and stage, freed on the stream after the kernel);
 * GS_ERR_CUDA if it cannot be allocated. */
gs_status ode_integrate_tableau(ode_rhs rhs, ode_tableau method, long n, double* x_dev,
                                const double* coef_dev, double t0, double dt, long nsteps,
                                void* stream);

/* Adams-Bashforth with `steps` = 1..8 steps (Table 1; Fig. 2c,d):
 * u_{m+1} = u_m + dt sum_{j<s} beta_j f(t_{m-j}, u_{m-j}) with the
 * Adams-Bashforth weights, t_m = t0 + m dt.  The first steps - 1 steps of a
 * call are one-step steps of order >= steps (RK4 for steps <= 4, the order-8
 * Fehlberg solution for 5..8), so the start-up does not limit the order; the
 * history lives in registers.  Same arguments and errors as
 * ode_integrate_tableau (the time-factor table: one value per step, plus the
 * start-up steps' stage times).  Enqueued on stream. */
gs_status ode_integrate_ab_steps(ode_rhs rhs, int steps, long n, double* x_dev, const double* coef_dev,
                                 double t0, double dt, long nsteps, void* stream);

/* Adams-Bashforth-Moulton with `steps` = 1..8 steps (Table 1), as a
 * predictor-corrector in PECE form (the paper names the method only; this
 * library's reading): with f_m = f(t_m, u_m),
 *   u* = u_m + dt sum_{j<s} beta_j f_{m-j}                (Adams-Bashforth)
 *   u_{m+1} = u_m + dt (beta*_0 f(t_{m+1}, u*) + sum_{1<=j<s} beta*_j f_{m+1-j})
 *                                                          (Adams-Moulton),
 * two evaluations of f per step, order s.  The first steps - 1 steps are
 * one-step steps of order >= steps as for ode_integrate_ab_steps.  The
 * Adams-Moulton weights are integrals of Lagrange basis polynomials,
 * evaluated on the host by Gauss-Legendre quadrature.  Same arguments and
 * errors as ode_integrate_ab_steps.  Enqueued on stream. */
gs_status ode_integrate_abm_steps(ode_rhs rhs, int steps, long n, double* x_dev, const double* coef_dev,
                                  double t0, double dt, long nsteps, void* stream);

/* Error-controlled integration of n INDEPENDENT scalar ODEs, each with its
 * own step size and controller (no global norm), from t0 to t_end with the
 * embedded pair `method` (ODE_TAB_DOPRI5, ODE_TAB_CK54, ODE_TAB_RKF78).
 * Per element: E = |err| / (atol + rtol (|x| + h |k1|)); E > 1 rejects and
 * shrinks dt = h max(0.9 E^(-1/(q-1)), 0.2); else accept, and if E < 0.5
 * grow dt = 0.9 h max(E, 5^-p)^(-1/p) (p, q = propagated / embedded order:
 * 5, 4 for Dormand-Prince and Cash-Karp, 8, 7 for Fehlberg); the last step
 * is clipped to t_end.  The powers E^(-1/k) are computed to a few ulps (an
 * FP32 estimate refined by two FP64 Newton steps), not by the correctly
 * rounded pow: step sizes can differ from a pow-based controller in the
 * last bits.  An element stops at t_end, after max_acc accepted
 * steps (< 0: no limit), after max_rej consecutive rejections or a step that
 * no longer advances t (GS_ERR_STEP_UNDERFLOW), on a non-finite error
 * (GS_ERR_NONFINITE) or after 2^22 attempts (GS_ERR_MAX_STEPS).  Optional
 * device outputs (each may be NULL): final t, next dt, accepted and rejected
 * counts, status per element.  INVALID: bad kind / method, n < 0,
 * non-finite t0 / t_end, dt0 <= 0, negative tolerances or both zero,
 * max_rej < 1.  Enqueued on stream.  (Fehlberg's embedded estimate is zero
 * for f = f(t), as for Eq. 1a/1b: its step size then only grows.) */
gs_status ode_integrate_adaptive_each(ode_rhs rhs, ode_tableau method, long n, double* x_dev,
                                      const double* coef_dev, double t0, double t_end, double dt0,
                                      double atol, double rtol, long max_acc, long max_rej,
                                      double* t_out_dev, double* dt_out_dev, long* n_acc_dev,
                                      long* n_rej_dev, int* status_dev, void* stream);


#ifdef __cplusplus
}
#endif
#endif /* GS_B300_H */
