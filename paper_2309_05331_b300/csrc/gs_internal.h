/*
 * gs_internal.h -- tuning, timing and test entry points of libgs_b300.so.
 *
 * These are exported by the library next to the calls of include/gs.h, but
 * they are not part of the method's interface: they pick kernel forms, tile
 * shapes and launch paths (every choice computes the same formulas), time
 * single kernels for the measurement, or let tests reach failure paths.
 * The benchmark, the tests, the project autotuner and the profiling helpers
 * use them.  Conventions (statuses, streams, ownership) are those of gs.h.
 */
#ifndef GS_B300_INTERNAL_H
#define GS_B300_INTERNAL_H

#include "../../include/gs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------- single-grid kernels ------------------------ */
/* Tile shape of the stencil kernels: a CTA of 32 x (ty+2) threads works on
 * columns of ty rows (30 cells wide in the generic kernel, 128 FP32 / 64 FP64
 * cells in the vectorised one) and owns an equal share, of at least zc
 * planes, of all columns' planes.  2 <= ty <= 14 (final kernels of the
 * generic and vectorised forms use at most 6), 0 <= zc <= 1024; zc = 0 (the default) lets every resident CTA
 * take a share (at least one plane).  Takes effect at the next integrator
 * call. */
gs_status gs_set_tile(gs_ctx* ctx, int ty, int zc);
gs_status gs_get_tile(const gs_ctx* ctx, int* ty, int* zc);

/* Stencil kernel form: 0 = automatic (a vectorised kernel when nx is a
 * multiple of its vector width, else the generic one; the autotuner may pick
 * per kernel), 1 = generic (one cell per thread, 30-cell rows), 2 =
 * vectorised (16-byte accesses: 4 FP32 or 2 FP64 cells per thread, 128- or
 * 64-cell rows per warp; the autotuner may still pick 8-byte rows), 3 =
 * vectorised 8-byte (FP32 only: 2 cells per thread, 64-cell rows), 4 =
 * staged (the 16-byte rows of form 2, with every thread copying its inputs
 * into a shared-memory ring 1 to 3 planes ahead with cp.async).  INVALID if
 * the form does not apply (nx not a multiple of the vector width).  All
 * forms compute the same formulas. */
gs_status gs_set_kernel_variant(gs_ctx* ctx, int variant);
/* The stencil kernel form the next call will use: 1 generic, 2 vectorised,
 * 4 staged. */
gs_status gs_get_kernel_variant(const gs_ctx* ctx, int* in_use);


/* Configuration in use for each Dormand-Prince kernel (index 0: k1, 1..6:
 * stages 2..7): form (1 generic, 2 vectorised 16-byte rows, 3 vectorised
 * 8-byte rows, 4 staged 16-byte rows), ty, zc.  Each argument: host array of 7 ints. */
gs_status gs_get_stage_configs(const gs_ctx* ctx, int* form, int* ty, int* zc);

/* Ring depth of the staged form (form 4): how many planes ahead each thread
 * copies its inputs, 1..3.  Sets the depth of every kernel (the autotuner
 * picks its own per kernel); a depth whose ring does not fit in shared
 * memory is reduced at launch.  gs_get_stage_depths: the depth each
 * Dormand-Prince kernel uses when it runs in form 4 (host array of 7 ints). */
/* Split of Dormand-Prince stages 6 and 7 (staged form): stage 6 also forms
 * the 5th-order solution y5 (b7 = 0, so y5 needs k1..k6 only), the error
 * terms of k1..k6 and the inverse error scale, and never stores k6; stage 7
 * evaluates k7 = F(y5) and adds its error term.  Two fewer field passes per
 * attempt (31 instead of 33).  mode: -1 automatic (on when the staged form
 * applies and no other kernel form is forced; the default), 0 off, 1 on
 * (INVALID if the staged form does not apply).  Same formulas, summed in
 * another order (y5 as (u + dt sum_{j<6} b_j k_j) + dt b6 k6).
 * gs_get_dopri5_split: 1 if the split is in use. */
/* Fixed-step RK4 (gs_step) on small grids in ONE cooperative launch: every
 * step's four stages run in a persistent kernel, separated by a grid
 * barrier, instead of four launches per step.  mode: -1 automatic (grids of
 * at most 2^18 cells; the default), 0 off, 1 on; ctas: the launch's CTA count
 * (0: automatic, at most what the GPU holds resident).  Same formulas and
 * summation order as the stage kernels.  A barrier wait that passes its
 * iteration limit makes gs_step return GS_ERR_CUDA.  gs_get_small_grid_path:
 * 1 if gs_step(GS_RK4) takes this path. */
gs_status gs_set_small_grid_path(gs_ctx* ctx, int mode, int ctas);
int gs_get_small_grid_path(const gs_ctx* ctx);
gs_status gs_set_dopri5_split(gs_ctx* ctx, int mode);
int gs_get_dopri5_split(const gs_ctx* ctx);

/* Dormand-Prince stages in pairs (Table 1 tableau; Eq. 2 right-hand side):
 * stages 2+3, 4+5 and 6+7 each run as ONE launch that computes the first
 * stage's k on the tile plus a one-cell ring (recomputed by neighbouring
 * tiles) and the second stage from it, so k2, k4 and k6 are never read back
 * and k6 is never stored.  Stages 2+3 also write the inverse error scale;
 * stages 4+5 write, instead of k4 and k5, stage 6's input Y6, y5 without
 * its k6 term and the error terms through k5 (the only combinations of k4
 * and k5 the later stages use); stages 6+7 read those and the scale, write y5 (the next state) and
 * k7 (the next k1), reduce the scaled error norm and run the controller: an
 * attempt moves 18 field passes instead of 31.  Requires the staged form (x
 * extent a multiple of the vector width); any ny, nz.  mode: -1 automatic
 * (on when the staged form applies and no other kernel form is forced;
 * gs_autotune keeps it on only if the pairs' summed kernel time beats the
 * single stages'), 0 off, 1 on (INVALID if the staged form does not apply).
 * The stage formulas are those of the single stages; Y_{i+1} is summed as
 * (u + dt sum_{j<i} a_{i+1,j} k_j) + dt a_{i+1,i} k_i; Y6 as u + ((the
 * k1..k3 part) + dt a64 k4 + dt a65 k5), y5 likewise plus dt b6 k6, and the
 * error terms as (the k1..k5 part) + dt e6 k6 + dt e7 k7.
 * gs_get_dopri5_fusion: 1 if the pairs are in use. */
gs_status gs_set_dopri5_fusion(gs_ctx* ctx, int mode);
int gs_get_dopri5_fusion(const gs_ctx* ctx);
/* The same switch runs fixed-step RK4 (gs_step, GS_RK4, on grids that do
 * not take the small-grid path) as two pair launches: k1 = F(u) and k2 =
 * F(u + dt/2 k1); then k3, k4 and the update u' = u + dt (k1/6 + k2/3 + k3/3
 * + k4/6) without storing k3 or k4: 7 field passes per step instead of 13.
 * Its automatic verdict is separate (gs_autotune times one RK4 step both
 * ways).  The update is summed as ((u + dt (k1/6 + k2/3)) + dt k3/3) + dt
 * k4/6.  gs_get_rk4_fusion: 1 if RK4 steps use the pairs. */
int gs_get_rk4_fusion(const gs_ctx* ctx);
/* Launch shape of pair kernel `pair` (0: Dormand-Prince stages 2+3, 1: 4+5,
 * 2: 6+7; 3: RK4 stages 1+2, 4: RK4 stages 3+4 with the update; -1: all
 * five): tile height ty (1..7 rows, 1..11 except for stages 4+5: the CTA
 * has ty + 5 warps, compiled for 12 warps up to 7 rows and for 16 above; -1
 * with ty > 7 is rejected) and input ring
 * depth (1..3 planes; cut back at launch to what shared memory holds).
 * gs_autotune overwrites it.  gs_get_pair_configs: host arrays of 5 ints. */
gs_status gs_set_pair_config(gs_ctx* ctx, int pair, int ty, int depth);
gs_status gs_get_pair_configs(const gs_ctx* ctx, int* ty, int* depth);
/* The ring depth each pair kernel launches with: its configured depth cut
 * back to what shared memory holds at its tile height (host array of 5). */
gs_status gs_get_pair_depths_in_use(const gs_ctx* ctx, int* depth);
gs_status gs_set_stage_depth(gs_ctx* ctx, int depth);
gs_status gs_get_stage_depths(const gs_ctx* ctx, int* depth);

/* Measurement aid: launches the kernels of one Dormand-Prince attempt of
 * the bound state one at a time between CUDA events on the context stream
 * and returns their average durations over `reps` repetitions (after one
 * warm-up): ms[0] = the k1 = F(u) kernel, ms[1..6] = stages 2..7 (stage 7
 * includes the error-norm reduction).  Outputs go to the context's scratch;
 * the bound state is not modified.  ms: host array of 7 doubles.
 * Synchronises. */
gs_status gs_time_stages(gs_ctx* ctx, int reps, double* ms);
/* Same for the pair kernels: ms[0] = k1, ms[1..3] = stages 2+3, 4+5, 6+7
 * (the last includes the error-norm reduction).  ms: host array of 4
 * doubles.  INVALID if the pair kernels do not apply.  Synchronises. */
gs_status gs_time_pairs(gs_ctx* ctx, int reps, double* ms);

/* Tile depth of the DC-PSE stage kernel: 0 (default: 4 where the grid has
 * fewer than 16 tiles of 8^3 per SM, else 8), 4 or 8; the results do not
 * depend on it.  INVALID: any other value. */
gs_status gs_set_dcpse_tile(gs_ctx* ctx, int tz);

/* ---------------------------- batched ensembles -------------------------- */
/* Segment shape: ty rows (2,4,6,8,14; stage 7 uses at most 6) of 32 cells,
 * zc planes (1..1024). */
gs_status gsb_set_tile(gsb_ctx* ctx, int ty, int zc);
/* Cache blocking by instance group: each attempt runs stages 2..7 over one
 * group of consecutive instances at a time, so a group's stage fields are
 * re-read from L2 instead of HBM.  cells_per_group: the group budget (a
 * group holds at least one instance); -1 = half the L2 over the working set
 * of a cell (state and stage fields, 20 values); 0 (the default) = one group
 * (every stage over all instances).  gsb_get_grouping: the budget in
 * use and the number of groups.  gsb_autotune also chooses the grouping. */
gs_status gsb_set_grouping(gsb_ctx* ctx, long long cells_per_group);
/* Segment code of the batched stage kernels: depth 1..3 = staged form (each
 * thread copies its inputs that many planes ahead into shared memory with
 * cp.async), 0 = vectorised form (direct loads; the default).  Same results.
 * gsb_autotune tunes the tile of the depth in use. */
gs_status gsb_set_stage_depth(gsb_ctx* ctx, int depth);
gs_status gsb_get_grouping(const gsb_ctx* ctx, long long* cells_per_group, int* ngroups);
/* Stage pairs for the batch: on = 1 runs each attempt as three pair steps
 * (stages 2+3, 4+5, 6+7; the single-grid pair segment), 18 field passes per
 * attempt instead of 33; ty = the tile height of the instances run with one
 * cell per lane (1..12; up to 7 in CTAs compiled for two per SM, 8..12 in
 * CTAs compiled for one), depth = the input ring depth (1..3, cut to what
 * shared memory holds).  The z-chunk is gsb_set_tile's.  Same formulas as
 * the single stages (results agree to rounding).  gsb_autotune_run tries
 * both forms.  gsb_get_pairs: the setting in use. */
gs_status gsb_set_pairs(gsb_ctx* ctx, int on, int ty, int depth);
gs_status gsb_get_pairs(const gsb_ctx* ctx, int* on, int* ty, int* depth);
/* Lane width of the stage pairs per instance: mode 1 (the default) gives
 * an instance 4 consecutive cells per lane (FP32, 16-byte rows: nx > 64 and
 * a multiple of 4) or 2 (8-byte FP32 / 16-byte FP64 rows: nx > 32 and even)
 * where every row starts on that boundary, one cell per lane otherwise; each
 * width runs its own launch per pair step over its instances, the wider
 * ones in 12-warp CTAs of tile height ty_wide (1..7).  mode 0: one cell per
 * lane for every instance.  Per-cell arithmetic is the same for every width
 * (FP64 results are identical).  gsb_get_pair_lanes: the setting and the
 * number of instances of width 1, 2 and 4 (host array of 3 ints). */
gs_status gsb_set_pair_lanes(gsb_ctx* ctx, int mode, int ty_wide);
gs_status gsb_get_pair_lanes(const gsb_ctx* ctx, int* mode, int* ty_wide, int* counts);

/* ---------------------------- learned surrogate -------------------------- */
/* Tensor-core engine of sur_conv3d (and of the network's convolutions),
 * process-wide: 0 = automatic (tcgen05 where it applies, else mma.sync),
 * 1 = warp-level mma.sync m16n8k16 for every shape, 2 = tcgen05 where it
 * applies.  The tcgen05 kernel covers 32 -> 32 and 8 -> 32 channels with
 * epi 0, 2 or 3 and 32 -> 8 channels with epi 1 or 3, on grids with
 * D % 4 == 0, H % 16 == 0, W % 8 == 0 (accumulators in tensor memory,
 * operands read from shared memory through matrix descriptors), and the
 * 32 x 32 weight gradient (sur_conv3d_wgrad) on grids with
 * H % 16 == 0, W % 8 == 0; other shapes always take mma.sync.  Both compute the same sums of exact
 * BF16 products in FP32 (summation order differs).  INVALID for other
 * values.  sur_conv_last_engine: 1 or 2, the engine of the last launch (0
 * before any).  sur_conv_tc_status: 1 if a tcgen05 launch of the layer primitives
 * (sur_conv3d, sur_conv3d_wgrad) gave up waiting for its MMAs, else 0 (the
 * kernel bounds every wait, frees its tensor memory and returns; from then
 * on the primitives return GS_ERR_CUDA). */
gs_status sur_set_conv_engine(int engine);
int sur_get_conv_engine(void);
int sur_conv_last_engine(void);
gs_status sur_conv_tc_status(unsigned int* timeouts);

/* Test hook for the failure path of the bounded tensor-core waits: sets the
 * timeout word of ctx (ctx = NULL: the layer primitives' word) to value, as
 * a tcgen05 kernel does when a wait gives up, so tests can check from the
 * host that every later call reports GS_ERR_CUDA (value 0 clears it).  No
 * GPU work is involved.  INVALID if the word was never allocated. */
gs_status sur_debug_set_timeout_word(sur_ctx* ctx, unsigned int value);

/* ---------------------------- pointwise ensembles ------------------------ */
/* The Adams-Moulton weights ode_integrate_abm_steps passes to its kernel
 * (host array of `steps` doubles, node t_{m+1} first), for the tests. */
gs_status ode_am_weights(int steps, double* w);

/* ---------------------------- measurement -------------------------------- */
/* Measures this device's FP64 fused-multiply-add throughput (TFLOP/s,
 * 2 flops per FMA) with independent dependent-chains; used as the ALU
 * roofline of the FP64 paths. Synchronises. */
gs_status gs_measure_fp64_peak(double* tflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GS_B300_INTERNAL_H */
