// gs_grid.cu -- single-grid Gray-Scott integrators behind the C ABI of gs.h.
//
// Every integrator is one CUDA graph: a conditional WHILE node whose body is
// the stage kernels of one step (RK4: 4, Dopri5: 6 after the first-same-as-
// last k1, Euler / Adams-Bashforth: 1).  The last kernel of the body advances
// the on-device control block (fixed-step counter, or the adaptive
// controller) and sets the loop condition, so the host enqueues one graph per
// call and reads the control block back once.
//
// Buffers: the caller's state (u, v) is state buffer 0; the context owns
// state buffer 1 and seven stage fields.  Which state buffer is current
// (and which k1 buffer, for Dopri5's first-same-as-last reuse) is a parity
// bit in the control block; if a run ends on buffer 1 a final kernel copies
// it back into the caller's arrays.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "gs_tile.cuh"
#include "gs_dcpse.cuh"
#include "gs_pair.cuh"
#include "gs_persist.cuh"
#include "gs_staged.cuh"
#include "gs_wide.cuh"
#include "tableaux.cuh"
#include "gs_internal.h"
#include "host_util.h"

using namespace gsk;

namespace {

enum GraphId { G_RK4 = 0, G_DOPRI5_FIXED, G_EULER, G_DOPRI5_ADAPT, G_AB4_START, G_AB4_MAIN, G_COUNT };

constexpr int kFields = 9;  // 0: second state buffer; 1..7: stage fields; 8: inverse error scale (split stages 6/7)

// Launch configuration of one stencil kernel.  form: 0 automatic, 1 generic
// (one cell per thread), 2 vectorised 16-byte rows (4 FP32 / 2 FP64 cells per
// thread), 3 vectorised 8-byte rows (2 FP32 cells per thread), 4 staged
// 16-byte rows (form 2 with the inputs copied into shared memory `depth`
// planes ahead).
struct KCfg {
    int form;
    int ty;
    int zc;
    int depth = 2;  // form 4 only: 1..kMaxDepth
};

}  // namespace

struct gs_ctx {
    gs_params p;
    long long N = 0;
    size_t esz = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int dev = 0, nsm = 0;
    void* state[2] = {nullptr, nullptr};
    unsigned char* scratch = nullptr;
    void* field[kFields][2] = {};
    DevCtrl* dctrl = nullptr;
    DevCtrl* hctrl = nullptr;     // pinned staging of the whole control block
    long long* hpatch = nullptr;  // pinned staging of single-field patches
    double* dlog = nullptr;
    long log_cap = 0;
    gs_observer obs = nullptr;  // user observer (gs_set_observer)
    void* obs_user = nullptr;
    KCfg def{0, 6, 0};      // kernels of RK4 / Euler / AB4 / F (form 0, zc 0: automatic)
    KCfg dp[7];             // Dormand-Prince k1 and stages 2..7 once tuned
    bool dp_tuned = false;
    int variant = 0;        // requested: 0 automatic, 1 generic, 2 vectorised, 3 vectorised 8-byte
    int split67 = -1;       // Dormand-Prince stages 6/7 split (MODE_DOPRI_S6/S7): -1 automatic, 0 off, 1 on
    int fuse = -1;          // Dormand-Prince stage pairs (2,3) (4,5) (6,7) in one launch each: -1 automatic, 0 off, 1 on
    bool fuse_auto = true;  // the automatic choice (the autotuner's verdict once tuned)
    bool rk4_fuse_auto = true;  // the automatic choice for RK4 (the autotuner's verdict once tuned)
    // pair kernels (tile height, ring depth): Dormand-Prince stages 2+3, 4+5,
    // 6+7; RK4 stages 1+2, 3+4
    KCfg pc[5] = {{5, 7, 0, 2}, {5, 7, 0, 2}, {5, 7, 0, 2}, {5, 7, 0, 2}, {5, 7, 0, 2}};
    int small_mode = -1;    // fixed-step RK4 in one cooperative launch: -1 automatic (small grids), 0 off, 1 on
    int small_ctas = 0;     // its CTA count (0: automatic)
    unsigned* pbar = nullptr;  // its grid barrier: u64 count, generation, error
    int lap = 0;               // Laplacian: 0 the 7-point stencil, 1 DC-PSE (gs_set_laplacian)
    double dcpse_rc = 0.0;
    int dcpse_count = 0;
    int dcpse_off[kDcpseMax][3] = {};
    double dcpse_w[kDcpseMax] = {};
    int dcpse_tz = 0;  // DC-PSE tile depth: 0 automatic, 4 or 8
    unsigned long long* demax = nullptr;  // tableau-path attempts: bits of the scaled error maximum
    // tableau path (DC-PSE Laplacian, or Cash-Karp / Fehlberg): stage fields
    // k8..k13 and a third stage-input buffer, allocated at first use
    unsigned char* tab_scratch = nullptr;
    void* tabx[7][2] = {};
    cudaGraph_t graph[G_COUNT] = {};
    cudaGraphExec_t exec[G_COUNT] = {};
    char err[512] = {0};
};

static void set_err(gs_ctx* c, cudaError_t e, const char* where) {
    if (c) snprintf(c->err, sizeof(c->err), "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            set_err(ctx, e_, #call);               \
            return GS_ERR_CUDA;                    \
        }                                          \
    } while (0)

// ---------------------------------------------------------------------------
// kernel launch helpers
// ---------------------------------------------------------------------------
template <typename T>
static Geom<T> make_geom(const gs_params& p) {
    Geom<T> g;
    g.nx = p.nx;
    g.ny = p.ny;
    g.nz = p.nz;
    const double hx = p.Lx / p.nx, hy = p.Ly / p.ny, hz = p.Lz / p.nz;
    g.cx = (T)(1.0 / (hx * hx));
    g.cy = (T)(1.0 / (hy * hy));
    g.cz = (T)(1.0 / (hz * hz));
    g.Du = (T)p.Du;
    g.Dv = (T)p.Dv;
    g.F = (T)p.F;
    g.k = (T)p.k;
    return g;
}

// vectorised form applicable: x-extent a multiple of the vector width
static bool form_ok(const gs_ctx* ctx, int form) {
    if (form == 1) return true;
    if (form == 2) return ctx->p.nx % (ctx->p.prec == GS_FP64 ? 2 : 4) == 0;
    if (form == 3) return ctx->p.prec == GS_FP32 && ctx->p.nx % 2 == 0;
    if (form == 4) return ctx->p.nx % (ctx->p.prec == GS_FP64 ? 2 : 4) == 0;
    return false;
}
static bool wide_ok(const gs_ctx* ctx) { return form_ok(ctx, 2) || form_ok(ctx, 3); }
// Dormand-Prince stages 6 and 7 split as MODE_DOPRI_S6 / S7 (staged form):
// automatic when the staged form applies and no other form is forced
static bool split67_on(const gs_ctx* ctx) {
    if (!form_ok(ctx, 4)) return false;
    if (ctx->split67 >= 0) return ctx->split67 == 1;
    return ctx->variant == 0 || ctx->variant == 4;
}
// Dormand-Prince stages as three pair launches (gs_pair.cuh): automatic when
// the staged form applies and no other form is forced (then the autotuner's
// verdict)
static bool pairs_on(const gs_ctx* ctx) {
    if (!form_ok(ctx, 4)) return false;
    if (ctx->fuse >= 0) return ctx->fuse == 1;
    return (ctx->variant == 0 || ctx->variant == 4) && ctx->fuse_auto;
}
// RK4 steps as two pair launches (same switch, its own automatic verdict)
static bool rk4_pairs_on(const gs_ctx* ctx) {
    if (!form_ok(ctx, 4)) return false;
    if (ctx->fuse >= 0) return ctx->fuse == 1;
    return (ctx->variant == 0 || ctx->variant == 4) && ctx->rk4_fuse_auto;
}
// the form a launch with configured form `form` actually uses
static int pick_form(const gs_ctx* ctx, int form) {
    if (ctx->variant == 1) return 1;
    if (ctx->variant == 3) return 3;
    if (ctx->variant == 4) return form_ok(ctx, 4) ? 4 : 1;
    if (form == 0) form = form_ok(ctx, 2) ? 2 : (form_ok(ctx, 3) ? 3 : 1);
    if (ctx->variant == 2 && form == 1) form = form_ok(ctx, 2) ? 2 : 3;
    if (!form_ok(ctx, form)) form = 1;
    return form;
}

// Grid and schedule of a stencil launch.  zc == 0 (automatic): if the
// columns fit in the resident CTAs, give each column k = min(nz, resident /
// columns) CTAs with one z-band each (column-split: all columns sweep the
// same planes together, no partial last wave); otherwise balanced linear
// shares over all resident CTAs.  zc > 0: balanced linear shares of at
// least zc planes.
static int plan_schedule(const gs_ctx* ctx, StageArgs& A, int occ) {
    const long long ncols = (long long)A.ntx * A.nty;
    const long long gmax_res = (long long)ctx->nsm * occ;
    const long long L = ncols * ctx->p.nz;
    A.kper = 0;
    if (A.zc == 0 && ncols <= gmax_res) {
        const long long k = std::min<long long>(ctx->p.nz, gmax_res / ncols);
        A.kper = (int)k;
        return (int)(k * ncols);
    }
    const long long g = std::max<long long>(1, A.zc > 0 ? L / A.zc : L);
    return (int)std::min<long long>(g, gmax_res);
}

template <typename T, int NK, int MODE, int VX>
static cudaError_t launch_wide(gs_ctx* ctx, cudaStream_t s, StageArgs A) {
    const Geom<T> g = make_geom<T>(ctx->p);
    auto kern = gs_stage_wide_kernel<T, NK, MODE, VX>;
    const int txw = 32 * VX;
    A.ntx = (ctx->p.nx + txw - 1) / txw;
    A.nty = (ctx->p.ny + A.ty - 1) / A.ty;
    const size_t smem = wide_smem_bytes<T, VX>(A.ty);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * (A.ty + 2), smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    // every CTA owns at least zc planes of the (column, z) space
    const int grid = plan_schedule(ctx, A, occ);
    kern<<<grid, dim3(32, A.ty + 2), smem, s>>>(g, A);
    return cudaGetLastError();
}

template <typename T, int NK, int MODE, int VX>
static cudaError_t launch_staged(gs_ctx* ctx, cudaStream_t s, StageArgs A, int depth) {
    const Geom<T> g = make_geom<T>(ctx->p);
    auto kern = gs_stage_staged_kernel<T, NK, MODE, VX>;
    const int txw = 32 * VX;
    A.ntx = (ctx->p.nx + txw - 1) / txw;
    A.nty = (ctx->p.ny + A.ty - 1) / A.ty;
    depth = std::max(1, std::min(depth, kMaxDepth));
    constexpr int NP = staged_pointwise<MODE>();
    size_t smem = staged_smem_bytes<T, NK, VX, NP>(A.ty, depth);
    // a deeper ring than shared memory holds is cut back
    while (depth > 1 && smem > kMaxSmemPerCta) smem = staged_smem_bytes<T, NK, VX, NP>(A.ty, --depth);
    if (smem > kMaxSmemPerCta) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * (A.ty + 2), smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const int grid = plan_schedule(ctx, A, occ);
    kern<<<grid, dim3(32, A.ty + 2), smem, s>>>(g, A, depth);
    return cudaGetLastError();
}

// the ring depth a pair launch uses: the requested one, cut back to what
// shared memory holds (leaving room for the kernel's static arrays)
constexpr size_t kPairSmemCap = kMaxSmemPerCta - 1024;
template <typename T, int NK, int MODE>
static int pair_depth_fit(int ty, int depth) {
    constexpr int VX = 16 / (int)sizeof(T);
    depth = std::max(1, std::min(depth, kMaxDepth));
    while (depth > 1 && pair_smem_bytes<T, NK, MODE, VX>(ty, depth) > kPairSmemCap) --depth;
    return depth;
}

template <typename T, int NK, int MODE, int VX>
static cudaError_t launch_pair(gs_ctx* ctx, cudaStream_t s, StageArgs A, int depth) {
    const Geom<T> g = make_geom<T>(ctx->p);
    if (A.ty < 1 || A.ty > pair_max_ty(MODE)) return cudaErrorInvalidConfiguration;
    auto kern = gs_pair_kernel<T, NK, MODE, VX, false>;
    if constexpr (MODE != MODE_PAIR_DOPRI45)
        if (A.ty > kPairMaxTY) kern = gs_pair_kernel<T, NK, MODE, VX, true>;
    const int txw = 32 * VX;
    A.ntx = (ctx->p.nx + txw - 1) / txw;
    A.nty = (ctx->p.ny + A.ty - 1) / A.ty;
    depth = pair_depth_fit<T, NK, MODE>(A.ty, depth);
    const size_t smem = pair_smem_bytes<T, NK, MODE, VX>(A.ty, depth);
    if (smem > kPairSmemCap) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * (A.ty + 5), smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const int grid = plan_schedule(ctx, A, occ);
    kern<<<grid, dim3(32, A.ty + 5), smem, s>>>(g, A, depth);
    return cudaGetLastError();
}

template <int NK, int MODE>
static cudaError_t launch_pair_nk(gs_ctx* ctx, cudaStream_t s, const StageArgs& A, const KCfg& cfg) {
    if (ctx->p.prec == GS_FP64) return launch_pair<double, NK, MODE, 2>(ctx, s, A, cfg.depth);
    return launch_pair<float, NK, MODE, 4>(ctx, s, A, cfg.depth);
}

template <typename T, int NK, int MODE>
static cudaError_t launch_generic(gs_ctx* ctx, cudaStream_t s, StageArgs A) {
    const Geom<T> g = make_geom<T>(ctx->p);
    auto kern = gs_stage_kernel<T, NK, MODE>;
    A.ntx = (ctx->p.nx + kTileX - 1) / kTileX;
    A.nty = (ctx->p.ny + A.ty - 1) / A.ty;
    const size_t smem = stage_smem_bytes<T>(A.ty);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * (A.ty + 2), smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const int grid = plan_schedule(ctx, A, occ);
    kern<<<grid, dim3(32, A.ty + 2), smem, s>>>(g, A);
    return cudaGetLastError();
}

template <typename T, int NK, int MODE>
static cudaError_t launch_stage_t(gs_ctx* ctx, cudaStream_t s, StageArgs A, int form, int depth) {
    if constexpr (MODE == MODE_DOPRI_S6 || MODE == MODE_DOPRI_S7) {
        // the split stages exist in the staged form only
        if (!form_ok(ctx, 4)) return cudaErrorInvalidConfiguration;
        return launch_staged<T, NK, MODE, 16 / sizeof(T)>(ctx, s, A, depth);
    }
    form = pick_form(ctx, form);
    if (form == 4) return launch_staged<T, NK, MODE, 16 / sizeof(T)>(ctx, s, A, depth);
    if (MODE != MODE_STAGE && A.ty > kMaxTYFinal) A.ty = kMaxTYFinal;
    if (form == 1) return launch_generic<T, NK, MODE>(ctx, s, A);
    if constexpr (sizeof(T) == 4) {
        if (form == 2) return launch_wide<T, NK, MODE, 4>(ctx, s, A);
        return launch_wide<T, NK, MODE, 2>(ctx, s, A);
    } else {
        return launch_wide<T, NK, MODE, 2>(ctx, s, A);
    }
}

template <int NK, int MODE>
static cudaError_t launch_stage_nk(gs_ctx* ctx, cudaStream_t s, const StageArgs& A, const KCfg& cfg) {
    if (ctx->p.prec == GS_FP64) return launch_stage_t<double, NK, MODE>(ctx, s, A, cfg.form, cfg.depth);
    return launch_stage_t<float, NK, MODE>(ctx, s, A, cfg.form, cfg.depth);
}

// Instantiated (NK, mode) pairs: stages with 0..5 inputs, final combinations
// with 0 (Euler, Adams-Bashforth) or 1 (RK4) halo inputs, Dormand-Prince
// stage 7 with 5.
static cudaError_t launch_stage(gs_ctx* ctx, cudaStream_t s, int nk, int mode, const StageArgs& A, const KCfg& cfg) {
    if (mode == MODE_STAGE) {
        switch (nk) {
            case 0: return launch_stage_nk<0, MODE_STAGE>(ctx, s, A, cfg);
            case 1: return launch_stage_nk<1, MODE_STAGE>(ctx, s, A, cfg);
            case 2: return launch_stage_nk<2, MODE_STAGE>(ctx, s, A, cfg);
            case 3: return launch_stage_nk<3, MODE_STAGE>(ctx, s, A, cfg);
            case 4: return launch_stage_nk<4, MODE_STAGE>(ctx, s, A, cfg);
            case 5: return launch_stage_nk<5, MODE_STAGE>(ctx, s, A, cfg);
            default: return cudaErrorInvalidValue;
        }
    }
    if (mode == MODE_FINAL) {
        if (nk == 0) return launch_stage_nk<0, MODE_FINAL>(ctx, s, A, cfg);
        if (nk == 1) return launch_stage_nk<1, MODE_FINAL>(ctx, s, A, cfg);
        return cudaErrorInvalidValue;
    }
    if (mode == MODE_DOPRI_S6) return nk == 5 ? launch_stage_nk<5, MODE_DOPRI_S6>(ctx, s, A, cfg) : cudaErrorInvalidValue;
    if (mode == MODE_DOPRI_S7) return nk == 0 ? launch_stage_nk<0, MODE_DOPRI_S7>(ctx, s, A, cfg) : cudaErrorInvalidValue;
    if (nk == 5) return launch_stage_nk<5, MODE_DOPRI_FINAL>(ctx, s, A, cfg);
    return cudaErrorInvalidValue;
}

static StageArgs base_args(gs_ctx* ctx, const KCfg& cfg) {
    StageArgs A;
    memset(&A, 0, sizeof(A));
    A.ty = cfg.ty;
    A.zc = cfg.zc;
    A.ctrl = ctx->dctrl;
    return A;
}
// configuration of Dormand-Prince kernel k (0: k1, 1..6: stages 2..7)
static const KCfg& dp_cfg(const gs_ctx* ctx, int k) { return ctx->dp_tuned ? ctx->dp[k] : ctx->def; }

// slot helpers over the context buffers
static Slot fld(gs_ctx* c, int f) { return slot_fixed(c->field[f][0], c->field[f][1]); }
static Slot state_sel(gs_ctx* c, int sel) {
    Slot s{};
    s.p[0][0] = c->state[0];
    s.p[0][1] = c->state[1];
    s.p[1][0] = c->field[0][0];
    s.p[1][1] = c->field[0][1];
    s.sel = sel;
    return s;
}
static Slot pair_sel(gs_ctx* c, int fa, int fb, int sel) {
    Slot s{};
    s.p[0][0] = c->field[fa][0];
    s.p[0][1] = c->field[fa][1];
    s.p[1][0] = c->field[fb][0];
    s.p[1][1] = c->field[fb][1];
    s.sel = sel;
    return s;
}
// Adams-Bashforth history ring over fields 1..4: f_m lives in field 1 + (m & 3)
static Slot ring(gs_ctx* c, int off) {
    Slot s{};
    for (int i = 0; i < 4; ++i) {
        s.p[i][0] = c->field[1 + i][0];
        s.p[i][1] = c->field[1 + i][1];
    }
    s.sel = SEL_RING;
    s.off = off;
    return s;
}

// ---------------------------------------------------------------------------
// Step bodies (enqueued on stream s; final kernel sets conditional h)
// ---------------------------------------------------------------------------
// RK4 with k-storage: k1 = F(u); k2 = F(u + dt/2 k1); k3 = F(u + dt/2 k2);
// u' = u + dt (k1/6 + k2/3 + k3/3 + k4/6) with k4 = F(u + dt k3).
// k1 goes to field 1 (or to the history ring when starting Adams-Bashforth).
// RK4 stage pair pi (3: k1 = F(u), k2 = F(u + dt/2 k1); 4: k3, k4 and the
// update u' = u + dt (k1/6 + k2/3 + k3/3 + k4/6) -> next state, controller)
static cudaError_t launch_rk4_pair(gs_ctx* ctx, cudaStream_t s, int pi, unsigned long long h, int use_cond) {
    const KCfg& cfg = ctx->pc[pi];
    StageArgs A = base_args(ctx, cfg);
    A.u = state_sel(ctx, SEL_CUR);
    A.has_out1 = 1;
    if (pi == 3) {
        A.bk[0] = 0.5;
        A.out0 = fld(ctx, 1);
        A.out1 = fld(ctx, 5);
        return launch_pair_nk<0, MODE_PAIR_STAGE>(ctx, s, A, cfg);
    }
    A.kin[0] = fld(ctx, 1);
    A.kin[1] = fld(ctx, 5);
    A.a[0] = 0.0;
    A.a[1] = 0.5;  // Y3 = u + dt/2 k2
    A.bk[0] = 0.0;
    A.bk[1] = 0.0;
    A.bk[2] = 1.0;  // Y4 = u + dt k3
    A.be[0] = 1.0 / 6.0;
    A.be[1] = 1.0 / 3.0;
    A.be[2] = 1.0 / 3.0;
    A.bf = 1.0 / 6.0;
    A.out0 = state_sel(ctx, SEL_NEXT);
    A.run_ctrl = 1;
    A.cond = h;
    A.use_cond = use_cond;
    return launch_pair_nk<2, MODE_PAIR_RK4>(ctx, s, A, cfg);
}

static cudaError_t body_rk4(gs_ctx* ctx, cudaStream_t s, unsigned long long h, int use_cond,
                            bool k1_in_ring) {
    if (!k1_in_ring && rk4_pairs_on(ctx)) {
        cudaError_t e = launch_rk4_pair(ctx, s, 3, h, use_cond);
        if (e != cudaSuccess) return e;
        return launch_rk4_pair(ctx, s, 4, h, use_cond);
    }
    const Slot k1 = k1_in_ring ? ring(ctx, 0) : fld(ctx, 1);
    StageArgs A = base_args(ctx, ctx->def);
    A.u = state_sel(ctx, SEL_CUR);
    A.out0 = k1;
    cudaError_t e = launch_stage(ctx, s, 0, MODE_STAGE, A, ctx->def);
    if (e != cudaSuccess) return e;
    A = base_args(ctx, ctx->def);
    A.u = state_sel(ctx, SEL_CUR);
    A.kin[0] = k1;
    A.a[0] = 0.5;
    A.out0 = fld(ctx, 5);
    if ((e = launch_stage(ctx, s, 1, MODE_STAGE, A, ctx->def)) != cudaSuccess) return e;
    A.kin[0] = fld(ctx, 5);
    A.out0 = fld(ctx, 6);
    if ((e = launch_stage(ctx, s, 1, MODE_STAGE, A, ctx->def)) != cudaSuccess) return e;
    A = base_args(ctx, ctx->def);
    A.u = state_sel(ctx, SEL_CUR);
    A.kin[0] = fld(ctx, 6);
    A.a[0] = 1.0;
    A.bk[0] = 1.0 / 3.0;
    A.ex[0] = k1;
    A.ex[1] = fld(ctx, 5);
    A.be[0] = 1.0 / 6.0;
    A.be[1] = 1.0 / 3.0;
    A.n_ex = 2;
    A.bf = 1.0 / 6.0;
    A.out0 = state_sel(ctx, SEL_NEXT);
    A.run_ctrl = 1;
    A.cond = h;
    A.use_cond = use_cond;
    return launch_stage(ctx, s, 1, MODE_FINAL, A, ctx->def);
}

static cudaError_t body_euler(gs_ctx* ctx, cudaStream_t s, unsigned long long h, int use_cond) {
    StageArgs A = base_args(ctx, ctx->def);
    A.u = state_sel(ctx, SEL_CUR);
    A.bf = 1.0;
    A.out0 = state_sel(ctx, SEL_NEXT);
    A.run_ctrl = 1;
    A.cond = h;
    A.use_cond = use_cond;
    return launch_stage(ctx, s, 0, MODE_FINAL, A, ctx->def);
}

// Adams-Bashforth 4 step m >= 3: f_m = F(u_m) into the ring,
// u_{m+1} = u_m + dt (55 f_m - 59 f_{m-1} + 37 f_{m-2} - 9 f_{m-3}) / 24.
static cudaError_t body_ab4(gs_ctx* ctx, cudaStream_t s, unsigned long long h, int use_cond) {
    StageArgs A = base_args(ctx, ctx->def);
    A.u = state_sel(ctx, SEL_CUR);
    A.bf = 55.0 / 24.0;
    A.ex[0] = ring(ctx, -1);
    A.ex[1] = ring(ctx, -2);
    A.ex[2] = ring(ctx, -3);
    A.be[0] = -59.0 / 24.0;
    A.be[1] = 37.0 / 24.0;
    A.be[2] = -9.0 / 24.0;
    A.n_ex = 3;
    A.out0 = state_sel(ctx, SEL_NEXT);
    A.out1 = ring(ctx, 0);
    A.has_out1 = 1;
    A.run_ctrl = 1;
    A.cond = h;
    A.use_cond = use_cond;
    return launch_stage(ctx, s, 0, MODE_FINAL, A, ctx->def);
}

// Dormand-Prince stage st (2..7) with k1 in the parity pair (fields 1, 2)
// and k2..k6 in fields 3..7; stage 7 writes y5 and k7 to the other buffers
// of their pairs and reduces the error norm.
static cudaError_t launch_dopri5_stage(gs_ctx* ctx, cudaStream_t s, int st, unsigned long long h,
                                       int use_cond) {
    const Slot k1 = pair_sel(ctx, 1, 2, SEL_CUR);
    const Slot k[7] = {k1, k1, fld(ctx, 3), fld(ctx, 4), fld(ctx, 5), fld(ctx, 6), fld(ctx, 7)};
    // k[i] = k_i for i = 1..6
    static const double A2[1] = {dp5::A21};
    static const double A3[2] = {dp5::A31, dp5::A32};
    static const double A4[3] = {dp5::A41, dp5::A42, dp5::A43};
    static const double A5[4] = {dp5::A51, dp5::A52, dp5::A53, dp5::A54};
    static const double A6[5] = {dp5::A61, dp5::A62, dp5::A63, dp5::A64, dp5::A65};
    static const double* rows[5] = {A2, A3, A4, A5, A6};
    const KCfg& cfg = dp_cfg(ctx, st - 1);
    StageArgs A = base_args(ctx, cfg);
    A.u = state_sel(ctx, SEL_CUR);
    if (split67_on(ctx) && st >= 6) {
        if (st == 6) {
            // k6 in registers only: y5 -> next state, error terms -> field 7,
            // inverse error scale -> field 8
            for (int j = 0; j < 5; ++j) {
                A.kin[j] = k[j + 1];
                A.a[j] = A6[j];
            }
            A.out0 = state_sel(ctx, SEL_NEXT);
            A.out1 = fld(ctx, 7);
            A.has_out1 = 1;
            A.out2 = fld(ctx, 8);
            return launch_stage(ctx, s, 5, MODE_DOPRI_S6, A, cfg);
        }
        A.u = state_sel(ctx, SEL_NEXT);  // y5
        A.ex[0] = fld(ctx, 7);
        A.ex[1] = fld(ctx, 8);
        A.n_ex = 2;
        A.out0 = pair_sel(ctx, 1, 2, SEL_NEXT);  // k7 = next k1
        A.run_ctrl = 1;
        A.cond = h;
        A.use_cond = use_cond;
        return launch_stage(ctx, s, 0, MODE_DOPRI_S7, A, cfg);
    }
    if (st < 7) {
        const int nk = st - 1;
        for (int j = 0; j < nk; ++j) {
            A.kin[j] = k[j + 1];
            A.a[j] = rows[st - 2][j];
        }
        A.out0 = k[st];
        return launch_stage(ctx, s, nk, MODE_STAGE, A, cfg);
    }
    A.kin[0] = k[1];
    A.kin[1] = k[3];
    A.kin[2] = k[4];
    A.kin[3] = k[5];
    A.kin[4] = k[6];
    A.a[0] = dp5::B1;
    A.a[1] = dp5::B3;
    A.a[2] = dp5::B4;
    A.a[3] = dp5::B5;
    A.a[4] = dp5::B6;
    A.out0 = state_sel(ctx, SEL_NEXT);
    A.out1 = pair_sel(ctx, 1, 2, SEL_NEXT);
    A.has_out1 = 1;
    A.run_ctrl = 1;
    A.cond = h;
    A.use_cond = use_cond;
    return launch_stage(ctx, s, 5, MODE_DOPRI_FINAL, A, cfg);
}

// Dormand-Prince stage pair pi (0: stages 2, 3 and the inverse error scale
// -> field 8; 1: stages 4, 5 -> stage 6's input Y6, P = y5 without its k6
// term and the error terms through k5 in fields 5..7; 2: stages 6, 7 from
// fields 5..8 with y5 -> next state, k7 -> next k1, the error norm and the
// controller)
static cudaError_t launch_dopri5_pair(gs_ctx* ctx, cudaStream_t s, int pi, unsigned long long h, int use_cond) {
    const Slot k1 = pair_sel(ctx, 1, 2, SEL_CUR);
    const Slot k[4] = {k1, k1, fld(ctx, 3), fld(ctx, 4)};  // k[i] = k_i
    const KCfg& cfg = ctx->pc[pi];
    StageArgs A = base_args(ctx, cfg);
    A.u = state_sel(ctx, SEL_CUR);
    A.has_out1 = 1;
    if (pi == 0) {
        A.kin[0] = k[1];
        A.a[0] = dp5::A21;
        A.bk[0] = dp5::A31;
        A.bk[1] = dp5::A32;
        A.out0 = k[2];
        A.out1 = k[3];
        A.out2 = fld(ctx, 8);  // inverse error scale
        return launch_pair_nk<1, MODE_PAIR_DOPRI23>(ctx, s, A, cfg);
    }
    if (pi == 1) {
        static const double a4[3] = {dp5::A41, dp5::A42, dp5::A43};
        static const double a5[4] = {dp5::A51, dp5::A52, dp5::A53, dp5::A54};
        for (int j = 0; j < 3; ++j) {
            A.kin[j] = k[j + 1];
            A.a[j] = a4[j];
        }
        for (int j = 0; j < 4; ++j) A.bk[j] = a5[j];
        A.out0 = fld(ctx, 5);  // Y6
        A.out1 = fld(ctx, 6);  // P
        A.out2 = fld(ctx, 7);  // error terms through k5
        return launch_pair_nk<3, MODE_PAIR_DOPRI45>(ctx, s, A, cfg);
    }
    A.u = fld(ctx, 5);
    A.kin[0] = fld(ctx, 6);
    A.kin[1] = fld(ctx, 7);
    A.kin[2] = fld(ctx, 8);
    A.out0 = state_sel(ctx, SEL_NEXT);       // y5
    A.out1 = pair_sel(ctx, 1, 2, SEL_NEXT);  // k7 = next k1
    A.run_ctrl = 1;
    A.cond = h;
    A.use_cond = use_cond;
    return launch_pair_nk<3, MODE_PAIR_DOPRI67>(ctx, s, A, cfg);
}

static cudaError_t body_dopri5(gs_ctx* ctx, cudaStream_t s, unsigned long long h, int use_cond) {
    if (pairs_on(ctx)) {
        for (int pi = 0; pi < 3; ++pi) {
            cudaError_t e = launch_dopri5_pair(ctx, s, pi, h, use_cond);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    for (int st = 2; st <= 7; ++st) {
        cudaError_t e = launch_dopri5_stage(ctx, s, st, h, use_cond);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// k1 = F(u) into the current k1 buffer (start of a Dormand-Prince run)
static cudaError_t launch_dopri5_k1(gs_ctx* ctx, cudaStream_t s) {
    const KCfg& cfg = dp_cfg(ctx, 0);
    StageArgs A = base_args(ctx, cfg);
    A.u = state_sel(ctx, SEL_CUR);
    A.out0 = pair_sel(ctx, 1, 2, SEL_CUR);
    return launch_stage(ctx, s, 0, MODE_STAGE, A, cfg);
}

static cudaError_t build_body(gs_ctx* ctx, int gid, cudaStream_t s, unsigned long long h, int use_cond) {
    switch (gid) {
        case G_RK4: return body_rk4(ctx, s, h, use_cond, false);
        case G_AB4_START: return body_rk4(ctx, s, h, use_cond, true);
        case G_EULER: return body_euler(ctx, s, h, use_cond);
        case G_AB4_MAIN: return body_ab4(ctx, s, h, use_cond);
        case G_DOPRI5_FIXED:
        case G_DOPRI5_ADAPT: return body_dopri5(ctx, s, h, use_cond);
        default: return cudaErrorInvalidValue;
    }
}

// The observer sees the state in the caller's buffers after the stream has
// drained; true: it asks to stop.
static bool observe(gs_ctx* ctx, double t, gs_status* st) {
    const cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        set_err(ctx, e, "observer: cudaStreamSynchronize");
        *st = GS_ERR_CUDA;
        return true;
    }
    return ctx->obs(t, ctx->state[0], ctx->state[1], ctx->obs_user) != 0;
}

// ---------------------------------------------------------------------------
// DC-PSE Laplacian (gs_dcpse.cuh): stencil from the moment conditions, and a
// host-driven stepping path (one stage kernel per stage; the last stage of a
// step or attempt also forms the new state and the error maximum).
// ---------------------------------------------------------------------------
// Weights of L f_p = sum_q w_q (f_{p+o_q} - f_p): for each axis d the kernel
// eta_d(z) = sum_g a_g z^g exp(-|z|^2) (z = -o_q, eps = h_d) with moments
// sum_q z_q^alpha eta_d(z_q) = 2 for alpha = 2 e_d and 0 for every other
// monomial of degree 1..3; the Gram system G a = m is symmetric positive
// definite and solved by Cholesky; w_q = sum_d eta_d(z_q) / h_d^2.
static bool dcpse_build(const double h[3], double rc, int off[][3], double* w, int* count) {
    int mono[19][3];
    int nm = 0;
    for (int deg = 1; deg <= 3; ++deg)
        for (int i = 0; i <= deg; ++i)
            for (int j = 0; i + j <= deg; ++j) {
                mono[nm][0] = i;
                mono[nm][1] = j;
                mono[nm][2] = deg - i - j;
                ++nm;
            }
    const int R = (int)std::floor(rc);
    int m = 0;
    for (int k = -R; k <= R; ++k)
        for (int j = -R; j <= R; ++j)
            for (int i = -R; i <= R; ++i) {
                if ((i | j | k) == 0 || (double)(i * i + j * j + k * k) > rc * rc) continue;
                if (m >= kDcpseMax) return false;
                off[m][0] = i;
                off[m][1] = j;
                off[m][2] = k;
                w[m] = 0.0;
                ++m;
            }
    if (m < nm) return false;
    auto monov = [&](const double z[3], int g) {
        double r = 1.0;
        for (int d = 0; d < 3; ++d)
            for (int e = 0; e < mono[g][d]; ++e) r *= z[d];
        return r;
    };
    for (int d = 0; d < 3; ++d) {
        double G[19][19] = {}, rhs[19];
        for (int g = 0; g < nm; ++g) rhs[g] = (mono[g][d] == 2 && mono[g][0] + mono[g][1] + mono[g][2] == 2) ? 2.0 : 0.0;
        for (int q = 0; q < m; ++q) {
            const double z[3] = {-(double)off[q][0], -(double)off[q][1], -(double)off[q][2]};
            const double ex = std::exp(-(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]));
            double ph[19];
            for (int g = 0; g < nm; ++g) ph[g] = monov(z, g);
            for (int a = 0; a < nm; ++a)
                for (int b = 0; b <= a; ++b) G[a][b] += ex * ph[a] * ph[b];
        }
        // Cholesky G = L L^T (lower triangle in place), then L y = rhs, L^T x = y
        for (int c = 0; c < nm; ++c) {
            double dsum = G[c][c];
            for (int k = 0; k < c; ++k) dsum -= G[c][k] * G[c][k];
            if (!(dsum > 0.0)) return false;
            G[c][c] = std::sqrt(dsum);
            for (int r = c + 1; r < nm; ++r) {
                double v = G[r][c];
                for (int k = 0; k < c; ++k) v -= G[r][k] * G[c][k];
                G[r][c] = v / G[c][c];
            }
        }
        double yv[19], coef[19];
        for (int r = 0; r < nm; ++r) {
            double v = rhs[r];
            for (int k = 0; k < r; ++k) v -= G[r][k] * yv[k];
            yv[r] = v / G[r][r];
        }
        for (int r = nm - 1; r >= 0; --r) {
            double v = yv[r];
            for (int k = r + 1; k < nm; ++k) v -= G[k][r] * coef[k];
            coef[r] = v / G[r][r];
        }
        for (int q = 0; q < m; ++q) {
            const double z[3] = {-(double)off[q][0], -(double)off[q][1], -(double)off[q][2]};
            const double ex = std::exp(-(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]));
            double eta = 0.0;
            for (int g = 0; g < nm; ++g) eta += coef[g] * monov(z, g);
            w[q] += eta * ex / (h[d] * h[d]);
        }
    }
    // the solution is even in the offset; make it exactly so (each pair
    // takes the mean of its two solved weights)
    for (int q = 0; q < m; ++q)
        for (int p = q + 1; p < m; ++p)
            if (off[p][0] == -off[q][0] && off[p][1] == -off[q][1] && off[p][2] == -off[q][2]) {
                const double wm = 0.5 * (w[q] + w[p]);
                w[q] = w[p] = wm;
            }
    *count = m;
    return true;
}

template <typename T>
static DcpseStencil<T> dcpse_stencil(const gs_ctx* ctx) {
    DcpseStencil<T> S;
    memset(&S, 0, sizeof(S));
    S.count = ctx->dcpse_count;
    double wsum = 0.0;
    for (int q = 0; q < S.count; ++q) {
        const int* o = ctx->dcpse_off[q];
        for (int d = 0; d < 3; ++d) S.off[q][d] = (signed char)o[d];
        S.w[q] = (T)ctx->dcpse_w[q];
        wsum += ctx->dcpse_w[q];
        // pairs {o, -o}: the representative has its last nonzero component positive
        const int lead = o[2] != 0 ? o[2] : (o[1] != 0 ? o[1] : o[0]);
        if (lead > 0) {
            S.pidx[S.npair] = (short)((o[2] * tile_edge(kDcpseR) + o[1]) * tile_edge(kDcpseR) + o[0]);
            S.pw[S.npair] = (T)ctx->dcpse_w[q];
            ++S.npair;
        }
    }
    S.wsum = (T)wsum;
    return S;
}

// The 7-point Laplacian as a stencil of the tableau path: the six
// neighbours with w = 1 / h_d^2 (and the centre through -sum w), halo 1.
template <typename T>
static DcpseStencil<T> seven_point_stencil(const gs_ctx* ctx) {
    DcpseStencil<T> S;
    memset(&S, 0, sizeof(S));
    const double h[3] = {ctx->p.Lx / ctx->p.nx, ctx->p.Ly / ctx->p.ny, ctx->p.Lz / ctx->p.nz};
    constexpr int E = tile_edge(1);
    double wsum = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double w = 1.0 / (h[d] * h[d]);
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            int o[3] = {0, 0, 0};
            o[d] = sgn;
            for (int k = 0; k < 3; ++k) S.off[S.count][k] = (signed char)o[k];
            S.w[S.count] = (T)w;
            ++S.count;
            wsum += w;
        }
        int o[3] = {0, 0, 0};
        o[d] = 1;
        S.pidx[S.npair] = (short)((o[2] * E + o[1]) * E + o[0]);
        S.pw[S.npair] = (T)w;
        ++S.npair;
    }
    S.wsum = (T)wsum;
    return S;
}

// one stage launch of the tableau path: tiles of 8 x 8 x 8 cells, or 8 x 8 x
// 4 where the grid has fewer than 16 deep tiles per SM (more, smaller CTAs
// even out the last wave; the deeper tile re-reads less halo); halo 3 for
// the DC-PSE stencil, 1 for the 7-point one
template <typename T, int R>
static cudaError_t tab_launch_r(gs_ctx* ctx, const DcpseStencil<T>& S, const DcpseStageArgs<T>& A) {
    const Geom<T> g = make_geom<T>(ctx->p);
    const long long tx = (ctx->p.nx + kDcpseT - 1) / kDcpseT, ty = (ctx->p.ny + kDcpseT - 1) / kDcpseT;
    const long long t8 = tx * ty * ((ctx->p.nz + 7) / 8);
    const int tz = ctx->dcpse_tz ? ctx->dcpse_tz : (t8 < 16LL * ctx->nsm ? 4 : 8);
    if (tz == 4) {
        const long long tiles = tx * ty * ((ctx->p.nz + 3) / 4);
        dcpse_stage_kernel<T, 4, R><<<(unsigned)tiles, 64 * 4, 0, ctx->stream>>>(g, S, A);
    } else {
        dcpse_stage_kernel<T, 8, R><<<(unsigned)t8, 64 * 8, 0, ctx->stream>>>(g, S, A);
    }
    return cudaGetLastError();
}
template <typename T>
static cudaError_t dcpse_launch(gs_ctx* ctx, const DcpseStageArgs<T>& A) {
    if (ctx->lap == 1) return tab_launch_r<T, kDcpseR>(ctx, dcpse_stencil<T>(ctx), A);
    return tab_launch_r<T, 1>(ctx, seven_point_stencil<T>(ctx), A);
}

// Butcher rows of the tableau path (tableaux.cuh): s stages, the orders p,
// q of the propagated / embedded solutions, error weights e = b - bhat.
struct HostTab {
    int s, p, q;
    double a[kTabMaxS][kTabMaxS];
    double b[kTabMaxS];
    double e[kTabMaxS];
};
template <class TB>
static HostTab tab_of() {
    HostTab T;
    memset(&T, 0, sizeof(T));
    T.s = TB::S;
    T.p = TB::P;
    T.q = TB::Q;
    for (int i = 0; i < TB::S; ++i) {
        for (int j = 0; j < i; ++j) T.a[i][j] = TB::a(i, j);
        T.b[i] = TB::b(i);
        T.e[i] = TB::Q > 0 ? TB::b(i) - TB::bh(i) : 0.0;
    }
    return T;
}
static HostTab host_tab(gs_method m) {
    switch (m) {
        case GS_EULER: return tab_of<TabEuler>();
        case GS_RK4: return tab_of<TabRK4>();
        case GS_CK54: return tab_of<TabCK54>();
        case GS_RKF78: return tab_of<TabRKF78>();
        case GS_MIDPOINT: return tab_of<TabMidpoint>();
        default: return tab_of<TabDP5>();
    }
}
static bool tab_method(gs_method m) { return m == GS_CK54 || m == GS_RKF78 || m == GS_MIDPOINT; }

// stage field k_j (1..13) and the third stage-input buffer (j = 14) of the
// tableau path
static void* tab_field(const gs_ctx* ctx, int j, int c) {
    if (j <= 7) return ctx->field[j][c];
    return ctx->tabx[j - 8][c];
}
static cudaError_t tab_ensure(gs_ctx* ctx) {
    if (!ctx->demax) {
        cudaError_t e = cudaMalloc(&ctx->demax, sizeof(unsigned long long));
        if (e != cudaSuccess) return e;
    }
    if (ctx->tab_scratch) return cudaSuccess;
    const size_t fbytes = ((size_t)ctx->N * ctx->esz + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&ctx->tab_scratch, fbytes * 2 * 7);
    if (e != cudaSuccess) {
        ctx->tab_scratch = nullptr;
        return e;
    }
    for (int f = 0; f < 7; ++f)
        for (int c = 0; c < 2; ++c) ctx->tabx[f][c] = ctx->tab_scratch + fbytes * (2 * f + c);
    return cudaSuccess;
}

// k = F(y) at every cell (the right-hand side, no further output)
template <typename T>
static cudaError_t dcpse_rhs(gs_ctx* ctx, void* const y[2], void* const out[2]) {
    DcpseStageArgs<T> A;
    memset(&A, 0, sizeof(A));
    for (int c = 0; c < 2; ++c) {
        A.y[c] = (const T*)y[c];
        A.u[c] = (const T*)y[c];
        A.out[c] = (T*)out[c];
    }
    return dcpse_launch<T>(ctx, A);
}

// out = u + dt sum_j b_j k_j; with emax, the attempt's scaled error maximum
template <typename T>
static cudaError_t dcpse_combine(gs_ctx* ctx, void* const u[2], int nk, const double* b, const double* e, double dt,
                                 double atol, double rtol, void* const out[2], bool err) {
    DcpseCombineArgs<T> A;
    memset(&A, 0, sizeof(A));
    for (int c = 0; c < 2; ++c) {
        A.u[c] = (const T*)u[c];
        A.out[c] = (T*)out[c];
        for (int j = 0; j < nk; ++j) A.k[j][c] = (const T*)tab_field(ctx, 1 + j, c);
    }
    for (int j = 0; j < nk; ++j) {
        A.b[j] = b[j];
        A.e[j] = e ? e[j] : 0.0;
    }
    A.nk = nk;
    A.dt = dt;
    A.atol = atol;
    A.rtol = rtol;
    A.emax = err ? ctx->demax : nullptr;
    const int blocks = (int)std::min<long long>((ctx->N + 255) / 256, (long long)ctx->nsm * 8);
    dcpse_combine_kernel<T><<<blocks, 256, 0, ctx->stream>>>(ctx->N, A);
    return cudaGetLastError();
}

// The stages of one step / attempt from state u: k_i into stage field i
// (1..s), the stage inputs Y_2..Y_s alternating between fields 8 and 0
// (Y_1 = u).
// With fin, the last stage also writes u + dt sum_j b_j k_j there and, with
// err, reduces the scaled error maximum into ctx->demax.  fin may be u
// itself when s_used > 1 (the last stage reads u at its own cells only).
template <typename T>
static cudaError_t dcpse_stages(gs_ctx* ctx, const HostTab& tab, int s_used, void* const u[2], double dt,
                                void* const* fin, bool err, double atol, double rtol) {
    void* const ybuf[2][2] = {{ctx->field[8][0], ctx->field[8][1]}, {ctx->field[0][0], ctx->field[0][1]}};
    for (int i = 0; i < s_used; ++i) {
        DcpseStageArgs<T> A;
        memset(&A, 0, sizeof(A));
        for (int c = 0; c < 2; ++c) {
            A.y[c] = (const T*)(i == 0 ? u[c] : ybuf[i % 2][c]);
            A.u[c] = (const T*)u[c];
            A.out[c] = (T*)tab_field(ctx, 1 + i, c);
            for (int j = 0; j < i; ++j) A.k[j][c] = (const T*)tab_field(ctx, 1 + j, c);
        }
        A.nk = i;
        A.dt = dt;
        if (i + 1 < s_used) {
            for (int j = 0; j <= i; ++j) A.an[j] = tab.a[i + 1][j];
            for (int c = 0; c < 2; ++c) A.yn[c] = (T*)ybuf[(i + 1) % 2][c];
        } else if (fin) {
            for (int j = 0; j <= i; ++j) {
                A.b[j] = tab.b[j];
                A.e[j] = tab.e[j];
            }
            for (int c = 0; c < 2; ++c) A.fin[c] = (T*)fin[c];
            A.atol = atol;
            A.rtol = rtol;
            A.emax = err ? ctx->demax : nullptr;
        }
        const cudaError_t e = dcpse_launch<T>(ctx, A);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
static gs_status dcpse_step(gs_ctx* ctx, gs_method method, double t0, double dt, long nsteps) {
    const HostTab tab = host_tab(method);
    if (tab.s > 7) CK(tab_ensure(ctx));
    // trailing stages with b = 0 (Dormand-Prince's stage 7) do not enter the solution
    int s_used = tab.s;
    while (s_used > 1 && tab.b[s_used - 1] == 0.0) --s_used;
    void* const u[2] = {ctx->state[0], ctx->state[1]};
    (void)t0;  // autonomous right-hand side
    for (long m = 0; m < nsteps; ++m) {
        if (s_used > 1) {
            CK(dcpse_stages<T>(ctx, tab, s_used, u, dt, u, false, 0.0, 0.0));
        } else {
            // one stage reads u with its halo: the update goes through its own pass
            CK(dcpse_stages<T>(ctx, tab, s_used, u, dt, nullptr, false, 0.0, 0.0));
            CK(dcpse_combine<T>(ctx, u, s_used, tab.b, nullptr, dt, 0.0, 0.0, u, false));
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return GS_OK;
}

// error-controlled integration with an embedded pair on the tableau path:
// the device computes the attempt and its error maximum, the host runs the
// controller of the graph path (same formulas and limits) with the pair's
// orders: reject dt = h max(0.9 E^(-1/(q-1)), 0.2), grow dt = 0.9 h
// max(E, 5^-p)^(-1/p)
template <typename T>
static gs_status dcpse_adaptive(gs_ctx* ctx, gs_method method, double atol, double rtol, double* t_io, double t_end,
                                double* dt_io, long max_acc, long* n_acc_out, long* n_rej_out) {
    const HostTab tab = host_tab(method);
    CK(tab_ensure(ctx));
    void* const u[2] = {ctx->state[0], ctx->state[1]};
    // the new state goes where the last stage does not read its input from
    // (field 0 holds the inputs of odd stage indices)
    const int flast = (tab.s - 1) % 2 == 1 ? 14 : 0;
    void* const ynew[2] = {flast ? tab_field(ctx, flast, 0) : ctx->field[0][0],
                           flast ? tab_field(ctx, flast, 1) : ctx->field[0][1]};
    const double grow_floor = std::pow(5.0, -(double)tab.p);
    const size_t bytes = ctx->esz * (size_t)ctx->N;
    double t = *t_io, dt = *dt_io;
    long long n_acc = 0, n_rej = 0, consec = 0, att = 0;
    gs_status status = GS_OK;
    std::vector<double> log;
    bool stop = ctx->obs && observe(ctx, t, &status);
    while (!stop && t < t_end && (max_acc < 0 || n_acc < max_acc)) {
        if (att >= kMaxAttempts) {
            status = GS_ERR_MAX_STEPS;
            break;
        }
        bool last = false;
        double h = dt;
        if (t + dt >= t_end) {
            h = t_end - t;
            last = true;
        }
        if (!(h > 0.0) || t + h == t) {
            status = GS_ERR_STEP_UNDERFLOW;
            break;
        }
        ++att;
        CK(cudaMemsetAsync(ctx->demax, 0, sizeof(unsigned long long), ctx->stream));
        CK(dcpse_stages<T>(ctx, tab, tab.s, u, h, ynew, true, atol, rtol));
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, ctx->demax, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        double E;
        memcpy(&E, &bits, sizeof(E));
        if (!std::isfinite(E)) {
            status = GS_ERR_NONFINITE;
            break;
        }
        if (E > 1.0) {
            ++n_rej;
            ++consec;
            dt = h * std::max(0.9 * std::pow(E, -1.0 / (double)(tab.q - 1)), 0.2);
            if (consec >= kMaxConsecutiveRejects) {
                status = GS_ERR_STEP_UNDERFLOW;
                break;
            }
            continue;
        }
        consec = 0;
        for (int c = 0; c < 2; ++c)
            CK(cudaMemcpyAsync(u[c], ynew[c], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        log.push_back(h);
        ++n_acc;
        t = last ? t_end : t + h;
        dt = E < 0.5 ? h * 0.9 * std::pow(std::max(E, grow_floor), -1.0 / (double)tab.p) : h;
        if (ctx->obs) stop = observe(ctx, t, &status);
    }
    // step log and counters where gs_get_step_log finds them
    const long nlog = (long)std::min<size_t>(log.size(), (size_t)ctx->log_cap);
    if (nlog > 0)
        CK(cudaMemcpyAsync(ctx->dlog, log.data(), sizeof(double) * (size_t)nlog, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    memset(ctx->hctrl, 0, sizeof(DevCtrl));
    ctx->hctrl->n_acc = n_acc;
    ctx->hctrl->n_rej = n_rej;
    *t_io = t;
    *dt_io = dt;
    if (n_acc_out) *n_acc_out = (long)n_acc;
    if (n_rej_out) *n_rej_out = (long)n_rej;
    return status;
}

static void drop_graphs(gs_ctx* ctx) {
    for (int i = 0; i < G_COUNT; ++i) {
        if (ctx->exec[i]) cudaGraphExecDestroy(ctx->exec[i]);
        if (ctx->graph[i]) cudaGraphDestroy(ctx->graph[i]);
        ctx->exec[i] = nullptr;
        ctx->graph[i] = nullptr;
    }
}

// WHILE(cond) { body } as an executable graph, cached per id.
static gs_status get_loop_graph(gs_ctx* ctx, int gid, cudaGraphExec_t* out) {
    if (ctx->exec[gid]) {
        *out = ctx->exec[gid];
        return GS_OK;
    }
    cudaGraph_t g = nullptr, body = nullptr;
    cudaGraphConditionalHandle h;
    cudaError_t e = make_while_graph(&g, &h, &body);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        set_err(ctx, e, "make_while_graph");
        return GS_ERR_CUDA;
    }
    e = cudaStreamBeginCaptureToGraph(ctx->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t eb = build_body(ctx, gid, ctx->cap, (unsigned long long)h, 1);
        cudaGraph_t tmp = body;
        e = cudaStreamEndCapture(ctx->cap, &tmp);
        if (eb != cudaSuccess) e = eb;
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        set_err(ctx, e, "capture of the step body");
        return GS_ERR_CUDA;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        set_err(ctx, e, "cudaGraphInstantiate");
        return GS_ERR_CUDA;
    }
    ctx->graph[gid] = g;
    ctx->exec[gid] = ex;
    *out = ex;
    return GS_OK;
}

// copy state buffer 1 back into the caller's arrays if the run ended there
template <typename T>
__global__ void copy_back_kernel(const DevCtrl* c, const T* __restrict__ a0, const T* __restrict__ a1,
                                 T* __restrict__ b0, T* __restrict__ b1, long long n) {
    if (c->parity == 0) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        b0[i] = a0[i];
        b1[i] = a1[i];
    }
}

static cudaError_t launch_copy_back(gs_ctx* ctx) {
    const int grid = ctx->nsm * 8;
    if (ctx->p.prec == GS_FP64)
        copy_back_kernel<double><<<grid, 256, 0, ctx->stream>>>(
            ctx->dctrl, (const double*)ctx->field[0][0], (const double*)ctx->field[0][1],
            (double*)ctx->state[0], (double*)ctx->state[1], ctx->N);
    else
        copy_back_kernel<float><<<grid, 256, 0, ctx->stream>>>(
            ctx->dctrl, (const float*)ctx->field[0][0], (const float*)ctx->field[0][1],
            (float*)ctx->state[0], (float*)ctx->state[1], ctx->N);
    return cudaGetLastError();
}

static gs_status upload_ctrl(gs_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->dctrl, ctx->hctrl, sizeof(DevCtrl), cudaMemcpyHostToDevice, ctx->stream));
    return GS_OK;
}

static gs_status download_ctrl_sync(gs_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->hctrl, ctx->dctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GS_OK;
}

static void init_fixed_ctrl(gs_ctx* ctx, double t0, double dt, long long limit) {
    DevCtrl* h = ctx->hctrl;
    memset(h, 0, sizeof(DevCtrl));
    h->mode = CTRL_FIXED;
    h->t = t0;
    h->t0 = t0;
    h->dt = dt;
    h->dt_try = dt;
    h->step_limit = limit;
    h->max_acc = -1;
    h->max_att = kMaxAttempts;
    h->t_end = INFINITY;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
// Grids up to this many cells keep their fields in L2: fixed-step RK4 then
// runs in one cooperative launch (gs_persist.cuh) by default.
constexpr long long kSmallGridCells = 1LL << 18;

template <typename T>
static gs_status rk4_persistent(gs_ctx* ctx, double dt, long nsteps) {
    auto kern = rk4_persistent_kernel<T>;
    const Geom<T> g = make_geom<T>(ctx->p);
    RK4Bufs<T> B;
    for (int c = 0; c < 2; ++c) {
        B.s[0][c] = static_cast<T*>(ctx->state[c]);
        B.s[1][c] = static_cast<T*>(ctx->field[0][c]);
        for (int j = 0; j < 3; ++j) B.k[j][c] = static_cast<T*>(ctx->field[1 + j][c]);
    }
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0));
    const long long want = ctx->small_ctas > 0 ? ctx->small_ctas : std::min<long long>(ctx->nsm, (ctx->N + 255) / 256);
    const int grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)ctx->nsm * std::max(occ, 1)));
    CK(cudaMemsetAsync(ctx->pbar, 0, 4 * sizeof(unsigned), ctx->stream));
    double dtv = dt;
    long long nst = nsteps;
    unsigned* bar = ctx->pbar;
    void* args[] = {(void*)&g, (void*)&B, (void*)&dtv, (void*)&nst, (void*)&bar};
    CK(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(256), args, 0, ctx->stream));
    unsigned err = 0;
    CK(cudaMemcpyAsync(&err, ctx->pbar + 3, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (err) {
        snprintf(ctx->err, sizeof(ctx->err), "rk4 persistent kernel: grid barrier wait expired");
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

static bool small_path(const gs_ctx* ctx) {
    if (ctx->N >= (1LL << 31)) return false;  // 32-bit cell indices
    if (ctx->small_mode >= 0) return ctx->small_mode == 1;
    return ctx->N <= kSmallGridCells;
}

extern "C" {

gs_status gs_create(const gs_params* p, void* stream, gs_ctx** out) {
    if (!p || !out) return GS_ERR_INVALID;
    *out = nullptr;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nx > 65535 || p->ny > 65535 || p->nz > 65535)
        return GS_ERR_INVALID;
    if (!(p->Lx > 0) || !(p->Ly > 0) || !(p->Lz > 0)) return GS_ERR_INVALID;
    if (p->prec != GS_FP64 && p->prec != GS_FP32) return GS_ERR_INVALID;
    gs_ctx* ctx = new (std::nothrow) gs_ctx();
    if (!ctx) return GS_ERR_NOMEM;
    ctx->p = *p;
    ctx->N = (long long)p->nx * p->ny * p->nz;
    ctx->esz = p->prec == GS_FP64 ? 8 : 4;
    ctx->stream = (cudaStream_t)stream;
    gs_status st = GS_OK;
    cudaError_t e;
    do {
        if ((e = cudaGetDevice(&ctx->dev)) != cudaSuccess) break;
        if ((e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->dev)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking)) != cudaSuccess) break;
        // one allocation: fields padded to 256 bytes
        const size_t fbytes = ((size_t)ctx->N * ctx->esz + 255) / 256 * 256;
        const size_t total = fbytes * 2 * kFields;
        if ((e = cudaMalloc(&ctx->scratch, total)) != cudaSuccess) {
            st = GS_ERR_NOMEM;
            break;
        }
        for (int f = 0; f < kFields; ++f)
            for (int c = 0; c < 2; ++c) ctx->field[f][c] = ctx->scratch + fbytes * (2 * f + c);
        if ((e = cudaMalloc(&ctx->dctrl, sizeof(DevCtrl))) != cudaSuccess) {
            st = GS_ERR_NOMEM;
            break;
        }
        if ((e = cudaMemset(ctx->dctrl, 0, sizeof(DevCtrl))) != cudaSuccess) break;
        if ((e = cudaMalloc(&ctx->pbar, 4 * sizeof(unsigned))) != cudaSuccess) {
            st = GS_ERR_NOMEM;
            break;
        }
        if ((e = cudaMallocHost(&ctx->hctrl, sizeof(DevCtrl))) != cudaSuccess) {
            st = GS_ERR_NOMEM;
            break;
        }
        if ((e = cudaMallocHost(&ctx->hpatch, 4 * sizeof(long long))) != cudaSuccess) {
            st = GS_ERR_NOMEM;
            break;
        }
        memset(ctx->hctrl, 0, sizeof(DevCtrl));
        ctx->def = KCfg{0, 6, 0};
    } while (0);
    if (e != cudaSuccess) {
        if (st == GS_OK) st = GS_ERR_CUDA;
        set_global_error(e, "gs_create");
        gs_destroy(ctx);
        return st;
    }
    *out = ctx;
    return GS_OK;
}

gs_status gs_destroy(gs_ctx* ctx) {
    if (!ctx) return GS_OK;
    drop_graphs(ctx);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->dctrl) cudaFree(ctx->dctrl);
    if (ctx->pbar) cudaFree(ctx->pbar);
    if (ctx->hctrl) cudaFreeHost(ctx->hctrl);
    if (ctx->hpatch) cudaFreeHost(ctx->hpatch);
    if (ctx->dlog) cudaFree(ctx->dlog);
    if (ctx->demax) cudaFree(ctx->demax);
    if (ctx->tab_scratch) cudaFree(ctx->tab_scratch);
    delete ctx;
    return GS_OK;
}

gs_status gs_bind_state(gs_ctx* ctx, void* u, void* v) {
    if (!ctx || !u || !v) return GS_ERR_INVALID;
    if (((uintptr_t)u & 15) || ((uintptr_t)v & 15)) return GS_ERR_INVALID;
    if (ctx->state[0] != u || ctx->state[1] != v) drop_graphs(ctx);
    ctx->state[0] = u;
    ctx->state[1] = v;
    return GS_OK;
}

gs_status gs_upload_state(gs_ctx* ctx, const void* uh, const void* vh) {
    if (!ctx || !uh || !vh || !ctx->state[0]) return GS_ERR_INVALID;
    const size_t bytes = (size_t)ctx->N * ctx->esz;
    CK(cudaMemcpyAsync(ctx->state[0], uh, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->state[1], vh, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return GS_OK;
}

gs_status gs_download_state(gs_ctx* ctx, void* uh, void* vh) {
    if (!ctx || !uh || !vh || !ctx->state[0]) return GS_ERR_INVALID;
    const size_t bytes = (size_t)ctx->N * ctx->esz;
    CK(cudaMemcpyAsync(uh, ctx->state[0], bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(vh, ctx->state[1], bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GS_OK;
}

gs_status gs_rhs(gs_ctx* ctx, double t, const void* u, const void* v, void* fu, void* fv) {
    (void)t;  // the Gray-Scott system is autonomous
    if (!ctx || !u || !v || !fu || !fv) return GS_ERR_INVALID;
    if (((uintptr_t)u | (uintptr_t)v | (uintptr_t)fu | (uintptr_t)fv) & 15) return GS_ERR_INVALID;
    StageArgs A = base_args(ctx, ctx->def);
    A.ctrl = nullptr;
    A.u = slot_fixed(const_cast<void*>(u), const_cast<void*>(v));
    A.out0 = slot_fixed(fu, fv);
    if (ctx->lap == 1) {
        void* const uu[2] = {const_cast<void*>(u), const_cast<void*>(v)};
        void* const out[2] = {fu, fv};
        CK(ctx->p.prec == GS_FP64 ? dcpse_rhs<double>(ctx, uu, out) : dcpse_rhs<float>(ctx, uu, out));
        return GS_OK;
    }
    CK(launch_stage(ctx, ctx->stream, 0, MODE_STAGE, A, ctx->def));
    return GS_OK;
}

gs_status gs_set_laplacian(gs_ctx* ctx, gs_laplacian kind, double rc_over_h) {
    if (!ctx) return GS_ERR_INVALID;
    if (kind == GS_LAP_7POINT) {
        drop_graphs(ctx);
        ctx->lap = 0;
        return GS_OK;
    }
    if (kind != GS_LAP_DCPSE || !(rc_over_h >= 2.0) || !(rc_over_h < 4.0)) return GS_ERR_INVALID;
    const double h[3] = {ctx->p.Lx / ctx->p.nx, ctx->p.Ly / ctx->p.ny, ctx->p.Lz / ctx->p.nz};
    int count = 0;
    if (!dcpse_build(h, rc_over_h, ctx->dcpse_off, ctx->dcpse_w, &count)) return GS_ERR_INVALID;
    if (!ctx->demax) CK(cudaMalloc(&ctx->demax, sizeof(unsigned long long)));
    drop_graphs(ctx);
    ctx->dcpse_count = count;
    ctx->dcpse_rc = rc_over_h;
    ctx->lap = 1;
    return GS_OK;
}

gs_status gs_set_observer(gs_ctx* ctx, gs_observer fn, void* user) {
    if (!ctx) return GS_ERR_INVALID;
    ctx->obs = fn;
    ctx->obs_user = fn ? user : nullptr;
    return GS_OK;
}

gs_status gs_set_dcpse_tile(gs_ctx* ctx, int tz) {
    if (!ctx || (tz != 0 && tz != 4 && tz != 8)) return GS_ERR_INVALID;
    ctx->dcpse_tz = tz;
    return GS_OK;
}

gs_status gs_get_dcpse_stencil(const gs_ctx* ctx, int* count, int* offsets, double* weights, int capacity) {
    if (!ctx || !count || ctx->lap != 1) return GS_ERR_INVALID;
    *count = ctx->dcpse_count;
    if (capacity < ctx->dcpse_count) return capacity == 0 ? GS_OK : GS_ERR_INVALID;
    if (!offsets || !weights) return GS_ERR_INVALID;
    for (int q = 0; q < ctx->dcpse_count; ++q) {
        for (int d = 0; d < 3; ++d) offsets[3 * q + d] = ctx->dcpse_off[q][d];
        weights[q] = ctx->dcpse_w[q];
    }
    return GS_OK;
}

gs_status gs_set_small_grid_path(gs_ctx* ctx, int mode, int ctas) {
    if (!ctx || mode < -1 || mode > 1 || ctas < 0 || ctas > 65535) return GS_ERR_INVALID;
    ctx->small_mode = mode;
    ctx->small_ctas = ctas;
    return GS_OK;
}

int gs_get_small_grid_path(const gs_ctx* ctx) { return ctx && small_path(ctx) ? 1 : 0; }

// Fixed steps with an observer: the step's loop graph runs one step per
// launch, the device control block carried from launch to launch (step
// limit raised, `done` cleared), so the step sequence, Dormand-Prince's
// first-same-as-last k1 and the Adams-Bashforth history are those of one
// uninterrupted run; after each step the state is copied to the caller's
// buffers and observed.
static gs_status step_observed(gs_ctx* ctx, gs_method method, double* t, double dt, long nsteps) {
    const double t0 = *t;
    gs_status st = GS_OK;
    if (observe(ctx, t0, &st)) return st;
    if (ctx->lap == 1 || tab_method(method)) {
        for (long n = 0; n < nsteps; ++n) {
            st = ctx->p.prec == GS_FP64 ? dcpse_step<double>(ctx, method, t0 + (double)n * dt, dt, 1)
                                        : dcpse_step<float>(ctx, method, t0 + (double)n * dt, dt, 1);
            if (st != GS_OK) return st;
            *t = t0 + (double)(n + 1) * dt;
            if (observe(ctx, *t, &st) && n + 1 < nsteps) return st;
        }
        return st;
    }
    const int gid = method == GS_RK4 ? G_RK4 : method == GS_EULER ? G_EULER : G_DOPRI5_FIXED;
    init_fixed_ctrl(ctx, t0, dt, 1);
    if ((st = upload_ctrl(ctx)) != GS_OK) return st;
    if (method == GS_DOPRI5) CK(launch_dopri5_k1(ctx, ctx->stream));
    for (long n = 0; n < nsteps; ++n) {
        if (n > 0) {
            ctx->hpatch[0] = n + 1;
            ctx->hpatch[1] = 0;
            CK(cudaMemcpyAsync(&ctx->dctrl->step_limit, &ctx->hpatch[0], sizeof(long long), cudaMemcpyHostToDevice,
                               ctx->stream));
            CK(cudaMemcpyAsync(&ctx->dctrl->done, &ctx->hpatch[1], sizeof(int), cudaMemcpyHostToDevice,
                               ctx->stream));
        }
        const int g = method == GS_AB4 ? (n < 3 ? G_AB4_START : G_AB4_MAIN) : gid;
        cudaGraphExec_t ex;
        if ((st = get_loop_graph(ctx, g, &ex)) != GS_OK) return st;
        CK(cudaGraphLaunch(ex, ctx->stream));
        CK(launch_copy_back(ctx));
        if ((st = download_ctrl_sync(ctx)) != GS_OK) return st;
        if (ctx->hctrl->status != GS_OK) return (gs_status)ctx->hctrl->status;
        *t = t0 + (double)(n + 1) * dt;
        if (ctx->obs(*t, ctx->state[0], ctx->state[1], ctx->obs_user) != 0 && n + 1 < nsteps) return GS_OK;
    }
    return GS_OK;
}

gs_status gs_step(gs_ctx* ctx, gs_method method, double* t, double dt, long nsteps) {
    if (!ctx || !t || !ctx->state[0] || nsteps < 0 || !std::isfinite(dt)) return GS_ERR_INVALID;
    if (method != GS_RK4 && method != GS_DOPRI5 && method != GS_AB4 && method != GS_EULER && !tab_method(method))
        return GS_ERR_INVALID;
    if (ctx->lap == 1 && method == GS_AB4) return GS_ERR_INVALID;
    if (nsteps == 0) return GS_OK;
    if (ctx->obs) return step_observed(ctx, method, t, dt, nsteps);
    const double t0 = *t;
    gs_status st;
    if (ctx->lap == 1 || tab_method(method)) {
        st = ctx->p.prec == GS_FP64 ? dcpse_step<double>(ctx, method, t0, dt, nsteps)
                                    : dcpse_step<float>(ctx, method, t0, dt, nsteps);
        if (st != GS_OK) return st;
        *t = t0 + (double)nsteps * dt;
        return GS_OK;
    }
    cudaGraphExec_t ex;
    if (method == GS_RK4 && small_path(ctx)) {
        st = ctx->p.prec == GS_FP64 ? rk4_persistent<double>(ctx, dt, nsteps) : rk4_persistent<float>(ctx, dt, nsteps);
        if (st != GS_OK) return st;
        *t = t0 + (double)nsteps * dt;
        return GS_OK;
    }
    if (method == GS_AB4) {
        const long long nstart = std::min<long long>(3, nsteps);
        init_fixed_ctrl(ctx, t0, dt, nstart);
        if ((st = upload_ctrl(ctx)) != GS_OK) return st;
        if ((st = get_loop_graph(ctx, G_AB4_START, &ex)) != GS_OK) return st;
        CK(cudaGraphLaunch(ex, ctx->stream));
        if (nsteps > 3) {
            // raise the step limit and clear `done` (own pinned staging: the
            // whole-block upload above may still be reading hctrl)
            ctx->hpatch[0] = nsteps;
            ctx->hpatch[1] = 0;
            CK(cudaMemcpyAsync(&ctx->dctrl->step_limit, &ctx->hpatch[0], sizeof(long long),
                               cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaMemcpyAsync(&ctx->dctrl->done, &ctx->hpatch[1], sizeof(int), cudaMemcpyHostToDevice,
                               ctx->stream));
            if ((st = get_loop_graph(ctx, G_AB4_MAIN, &ex)) != GS_OK) return st;
            CK(cudaGraphLaunch(ex, ctx->stream));
        }
    } else {
        const int gid = method == GS_RK4 ? G_RK4 : method == GS_EULER ? G_EULER : G_DOPRI5_FIXED;
        init_fixed_ctrl(ctx, t0, dt, nsteps);
        if ((st = upload_ctrl(ctx)) != GS_OK) return st;
        if (method == GS_DOPRI5) CK(launch_dopri5_k1(ctx, ctx->stream));
        if ((st = get_loop_graph(ctx, gid, &ex)) != GS_OK) return st;
        CK(cudaGraphLaunch(ex, ctx->stream));
    }
    CK(launch_copy_back(ctx));
    if ((st = download_ctrl_sync(ctx)) != GS_OK) return st;
    *t = t0 + (double)nsteps * dt;
    return GS_OK;
}

gs_status gs_integrate_adaptive(gs_ctx* ctx, double atol, double rtol, double* t, double t_end,
                                double* dt, long max_accepted, long* n_accepted, long* n_rejected) {
    if (!ctx || !t || !dt || !ctx->state[0]) return GS_ERR_INVALID;
    if (!(atol >= 0) || !(rtol >= 0) || !(atol > 0 || rtol > 0) || !(*dt > 0) || std::isnan(t_end))
        return GS_ERR_INVALID;
    if (n_accepted) *n_accepted = 0;
    if (n_rejected) *n_rejected = 0;
    if (!(*t < t_end) || max_accepted == 0) return GS_OK;
    if (ctx->lap == 1)
        return ctx->p.prec == GS_FP64 ? dcpse_adaptive<double>(ctx, GS_DOPRI5, atol, rtol, t, t_end, dt, max_accepted,
                                                               n_accepted, n_rejected)
                                      : dcpse_adaptive<float>(ctx, GS_DOPRI5, atol, rtol, t, t_end, dt, max_accepted,
                                                              n_accepted, n_rejected);
    const bool obs = ctx->obs != nullptr;
    gs_status st = GS_OK;
    if (obs && observe(ctx, *t, &st)) return st;
    DevCtrl* h = ctx->hctrl;
    memset(h, 0, sizeof(DevCtrl));
    h->mode = CTRL_ADAPTIVE;
    h->t = *t;
    h->t0 = *t;
    h->t_end = t_end;
    h->dt = *dt;
    h->atol = atol;
    h->rtol = rtol;
    // with an observer the loop graph stops after every accepted step
    h->max_acc = obs ? 1 : (max_accepted < 0 ? -1 : max_accepted);
    h->max_att = kMaxAttempts;
    h->log_dt = ctx->dlog;
    h->log_cap = ctx->log_cap;
    double ht = *dt;
    if (h->t + ht >= t_end) {
        ht = t_end - h->t;
        h->last = 1;
    }
    if (!(ht > 0.0) || h->t + ht == h->t) return GS_ERR_STEP_UNDERFLOW;
    h->dt_try = ht;
    if ((st = upload_ctrl(ctx)) != GS_OK) return st;
    CK(launch_dopri5_k1(ctx, ctx->stream));
    cudaGraphExec_t ex;
    if ((st = get_loop_graph(ctx, G_DOPRI5_ADAPT, &ex)) != GS_OK) return st;
    for (;;) {
        CK(cudaGraphLaunch(ex, ctx->stream));
        CK(launch_copy_back(ctx));
        if ((st = download_ctrl_sync(ctx)) != GS_OK) return st;
        if (!obs || h->status != GS_OK) break;
        const bool stop = ctx->obs(h->t, ctx->state[0], ctx->state[1], ctx->obs_user) != 0;
        if (stop || !(h->t < t_end) || (max_accepted >= 0 && h->n_acc >= max_accepted)) break;
        // the next attempt, prepared as the device controller prepares it
        // when it continues (the control block is the device's own copy)
        if (h->n_att >= h->max_att) {
            h->status = GS_ERR_MAX_STEPS;
            break;
        }
        ht = h->dt;
        h->last = 0;
        if (h->t + ht >= t_end) {
            ht = t_end - h->t;
            h->last = 1;
        }
        if (!(ht > 0.0) || h->t + ht == h->t) {
            h->status = GS_ERR_STEP_UNDERFLOW;
            break;
        }
        h->dt_try = ht;
        h->max_acc = h->n_acc + 1;
        h->done = 0;
        if ((st = upload_ctrl(ctx)) != GS_OK) return st;
    }
    *t = h->t;
    *dt = h->dt;
    if (n_accepted) *n_accepted = (long)h->n_acc;
    if (n_rejected) *n_rejected = (long)h->n_rej;
    return (gs_status)h->status;
}

gs_status gs_integrate_adaptive_pair(gs_ctx* ctx, gs_method pair, double atol, double rtol, double* t, double t_end,
                                     double* dt, long max_accepted, long* n_accepted, long* n_rejected) {
    if (pair == GS_DOPRI5)
        return gs_integrate_adaptive(ctx, atol, rtol, t, t_end, dt, max_accepted, n_accepted, n_rejected);
    if (!ctx || !t || !dt || !ctx->state[0] || (pair != GS_CK54 && pair != GS_RKF78)) return GS_ERR_INVALID;
    if (!(atol >= 0) || !(rtol >= 0) || !(atol > 0 || rtol > 0) || !(*dt > 0) || std::isnan(t_end))
        return GS_ERR_INVALID;
    if (n_accepted) *n_accepted = 0;
    if (n_rejected) *n_rejected = 0;
    if (!(*t < t_end) || max_accepted == 0) return GS_OK;
    return ctx->p.prec == GS_FP64
               ? dcpse_adaptive<double>(ctx, pair, atol, rtol, t, t_end, dt, max_accepted, n_accepted, n_rejected)
               : dcpse_adaptive<float>(ctx, pair, atol, rtol, t, t_end, dt, max_accepted, n_accepted, n_rejected);
}

gs_status gs_set_step_log(gs_ctx* ctx, long capacity) {
    if (!ctx || capacity < 0) return GS_ERR_INVALID;
    if (ctx->dlog) {
        CK(cudaFree(ctx->dlog));
        ctx->dlog = nullptr;
    }
    ctx->log_cap = 0;
    if (capacity > 0) {
        CK(cudaMalloc(&ctx->dlog, sizeof(double) * (size_t)capacity));
        ctx->log_cap = capacity;
    }
    return GS_OK;
}

gs_status gs_get_step_log(gs_ctx* ctx, double* dts, long capacity, long* count) {
    if (!ctx || capacity < 0 || (capacity > 0 && !dts)) return GS_ERR_INVALID;
    const long n = (long)ctx->hctrl->n_acc;
    if (count) *count = n;
    const long m = std::min(std::min(n, capacity), ctx->log_cap);
    if (m > 0) {
        CK(cudaMemcpyAsync(dts, ctx->dlog, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return GS_OK;
}

gs_status gs_set_tile(gs_ctx* ctx, int ty, int zc) {
    if (!ctx) return GS_ERR_INVALID;
    if (ty < 2 || ty > kMaxTY || zc < 0 || zc > 1024)
        return GS_ERR_INVALID;
    drop_graphs(ctx);
    ctx->def.ty = ty;
    ctx->def.zc = zc;
    ctx->dp_tuned = false;  // an explicit tile applies to every kernel
    return GS_OK;
}

gs_status gs_get_tile(const gs_ctx* ctx, int* ty, int* zc) {
    if (!ctx || !ty || !zc) return GS_ERR_INVALID;
    *ty = ctx->def.ty;
    *zc = ctx->def.zc;
    return GS_OK;
}

gs_status gs_set_kernel_variant(gs_ctx* ctx, int variant) {
    if (!ctx || variant < 0 || variant > 4) return GS_ERR_INVALID;
    if (variant == 2 && !wide_ok(ctx)) return GS_ERR_INVALID;
    if (variant == 3 && !form_ok(ctx, 3)) return GS_ERR_INVALID;
    if (variant == 4 && !form_ok(ctx, 4)) return GS_ERR_INVALID;
    drop_graphs(ctx);
    ctx->variant = variant;
    return GS_OK;
}

gs_status gs_get_kernel_variant(const gs_ctx* ctx, int* in_use) {
    if (!ctx || !in_use) return GS_ERR_INVALID;
    const int f = pick_form(ctx, ctx->def.form);
    *in_use = f == 1 ? 1 : (f == 4 ? 4 : 2);
    return GS_OK;
}

gs_status gs_set_dopri5_split(gs_ctx* ctx, int mode) {
    if (!ctx || mode < -1 || mode > 1) return GS_ERR_INVALID;
    if (mode == 1 && !form_ok(ctx, 4)) return GS_ERR_INVALID;
    drop_graphs(ctx);
    ctx->split67 = mode;
    return GS_OK;
}

int gs_get_dopri5_split(const gs_ctx* ctx) { return ctx && split67_on(ctx) ? 1 : 0; }

gs_status gs_set_dopri5_fusion(gs_ctx* ctx, int mode) {
    if (!ctx || mode < -1 || mode > 1) return GS_ERR_INVALID;
    if (mode == 1 && !form_ok(ctx, 4)) return GS_ERR_INVALID;
    drop_graphs(ctx);
    ctx->fuse = mode;
    return GS_OK;
}

int gs_get_dopri5_fusion(const gs_ctx* ctx) { return ctx && pairs_on(ctx) ? 1 : 0; }

// the launch mode of pair kernel pi (0..2: Dormand-Prince 2+3, 4+5, 6+7;
// 3, 4: RK4 1+2, 3+4)
static int pair_mode(int pi) {
    switch (pi) {
        case 0: return MODE_PAIR_DOPRI23;
        case 1: return MODE_PAIR_DOPRI45;
        case 2: return MODE_PAIR_DOPRI67;
        case 4: return MODE_PAIR_RK4;
        default: return MODE_PAIR_STAGE;
    }
}

gs_status gs_set_pair_config(gs_ctx* ctx, int pair, int ty, int depth) {
    if (!ctx || pair < -1 || pair > 4 || ty < 1 || depth < 1 || depth > kMaxDepth) return GS_ERR_INVALID;
    for (int pi = 0; pi < 5; ++pi)
        if ((pair < 0 || pair == pi) && ty > pair_max_ty(pair_mode(pi))) return GS_ERR_INVALID;
    drop_graphs(ctx);
    for (int pi = 0; pi < 5; ++pi)
        if (pair < 0 || pair == pi) ctx->pc[pi] = KCfg{5, ty, 0, depth};
    return GS_OK;
}

int gs_get_rk4_fusion(const gs_ctx* ctx) { return ctx && rk4_pairs_on(ctx) ? 1 : 0; }

gs_status gs_get_pair_configs(const gs_ctx* ctx, int* ty, int* depth) {
    if (!ctx || !ty || !depth) return GS_ERR_INVALID;
    for (int pi = 0; pi < 5; ++pi) {
        ty[pi] = ctx->pc[pi].ty;
        depth[pi] = ctx->pc[pi].depth;
    }
    return GS_OK;
}

gs_status gs_get_pair_depths_in_use(const gs_ctx* ctx, int* depth) {
    if (!ctx || !depth) return GS_ERR_INVALID;
    const bool f64 = ctx->p.prec == GS_FP64;
    for (int pi = 0; pi < 5; ++pi) {
        const int ty = ctx->pc[pi].ty, d = ctx->pc[pi].depth;
        if (pi == 3)
            depth[pi] = f64 ? pair_depth_fit<double, 0, MODE_PAIR_STAGE>(ty, d)
                            : pair_depth_fit<float, 0, MODE_PAIR_STAGE>(ty, d);
        else if (pi == 4)
            depth[pi] = f64 ? pair_depth_fit<double, 2, MODE_PAIR_RK4>(ty, d)
                            : pair_depth_fit<float, 2, MODE_PAIR_RK4>(ty, d);
        else if (pi == 0)
            depth[pi] = f64 ? pair_depth_fit<double, 1, MODE_PAIR_DOPRI23>(ty, d)
                            : pair_depth_fit<float, 1, MODE_PAIR_DOPRI23>(ty, d);
        else if (pi == 1)
            depth[pi] = f64 ? pair_depth_fit<double, 3, MODE_PAIR_DOPRI45>(ty, d)
                            : pair_depth_fit<float, 3, MODE_PAIR_DOPRI45>(ty, d);
        else
            depth[pi] = f64 ? pair_depth_fit<double, 3, MODE_PAIR_DOPRI67>(ty, d)
                            : pair_depth_fit<float, 3, MODE_PAIR_DOPRI67>(ty, d);
    }
    return GS_OK;
}

gs_status gs_set_stage_depth(gs_ctx* ctx, int depth) {
    if (!ctx || depth < 1 || depth > kMaxDepth) return GS_ERR_INVALID;
    drop_graphs(ctx);
    ctx->def.depth = depth;
    for (int k = 0; k < 7; ++k) ctx->dp[k].depth = depth;
    return GS_OK;
}

gs_status gs_get_stage_depths(const gs_ctx* ctx, int* depth) {
    if (!ctx || !depth) return GS_ERR_INVALID;
    for (int k = 0; k < 7; ++k) depth[k] = dp_cfg(ctx, k).depth;
    return GS_OK;
}

gs_status gs_get_stage_configs(const gs_ctx* ctx, int* form, int* ty, int* zc) {
    if (!ctx || !form || !ty || !zc) return GS_ERR_INVALID;
    for (int k = 0; k < 7; ++k) {
        const KCfg& c = dp_cfg(ctx, k);
        form[k] = (k >= 5 && split67_on(ctx)) ? 4 : pick_form(ctx, c.form);
        ty[k] = (k == 6 && form[k] != 4 && c.ty > kMaxTYFinal) ? kMaxTYFinal : c.ty;
        zc[k] = c.zc;
    }
    return GS_OK;
}

// time one Dormand-Prince kernel k (0: k1, 1..6: stages 2..7) with the
// configuration currently in ctx->dp[k], from a fixed control block (parity 0)
static gs_status time_dp_kernel(gs_ctx* ctx, int k, int reps, cudaEvent_t e0, cudaEvent_t e1, float* ms_out) {
    float acc = 0.f;
    for (int r = 0; r < reps + 1; ++r) {
        init_fixed_ctrl(ctx, 0.0, 1e-3, 1 << 30);
        gs_status st = upload_ctrl(ctx);
        if (st != GS_OK) return st;
        CK(cudaEventRecord(e0, ctx->stream));
        cudaError_t e = (k == 0) ? launch_dopri5_k1(ctx, ctx->stream)
                                 : launch_dopri5_stage(ctx, ctx->stream, k + 1, 0, 0);
        if (e != cudaSuccess) {
            set_err(ctx, e, "autotune launch");
            return GS_ERR_CUDA;
        }
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0) acc += ms;  // the first launch is a warm-up
    }
    *ms_out = acc / reps;
    return GS_OK;
}

// time Dormand-Prince pair kernel pi with the configuration in ctx->pc[pi]
static gs_status time_pair_kernel(gs_ctx* ctx, int pi, int reps, cudaEvent_t e0, cudaEvent_t e1, float* ms_out) {
    float acc = 0.f;
    for (int r = 0; r < reps + 1; ++r) {
        init_fixed_ctrl(ctx, 0.0, 1e-3, 1 << 30);
        gs_status st = upload_ctrl(ctx);
        if (st != GS_OK) return st;
        CK(cudaEventRecord(e0, ctx->stream));
        cudaError_t e = pi < 3 ? launch_dopri5_pair(ctx, ctx->stream, pi, 0, 0) : launch_rk4_pair(ctx, ctx->stream, pi, 0, 0);
        if (e != cudaSuccess) {
            set_err(ctx, e, "autotune launch");
            return GS_ERR_CUDA;
        }
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0) acc += ms;
    }
    *ms_out = acc / reps;
    return GS_OK;
}

gs_status gs_autotune(gs_ctx* ctx, int* ty_out, int* zc_out, double* best_ms) {
    if (!ctx || !ctx->state[0]) return GS_ERR_INVALID;
    static const int cand[][2] = {{2, 0}, {4, 0}, {6, 0}, {8, 0}, {14, 0}, {4, 4}, {6, 4}, {8, 4}, {6, 16}, {8, 16}};
    // the staged form: every tile height (the column-split schedule fills
    // the resident CTAs best at a height that depends on the grid) x ring
    // depth 1 or 2 (a third plane in flight never paid for its shared memory)
    int forms[4], nf = 0;
    for (int f = 1; f <= 4; ++f) {
        if (!form_ok(ctx, f)) continue;
        if (ctx->variant == 1 && f != 1) continue;
        if (ctx->variant == 2 && f == 1) continue;
        if (ctx->variant == 3 && f != 3) continue;
        if (ctx->variant == 4 && f != 4) continue;
        forms[nf++] = f;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    drop_graphs(ctx);
    // realistic stage inputs: one full attempt with the current configuration
    gs_status st = GS_OK;
    for (int k = 0; k < 7 && st == GS_OK; ++k) {
        float ms;
        st = time_dp_kernel(ctx, k, 1, e0, e1, &ms);
    }
    KCfg best_cfg[7];
    float total = 0.f, stage_best[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 7 && st == GS_OK; ++k) {
        float best = 1e30f;
        best_cfg[k] = dp_cfg(ctx, k);
        const KCfg saved = ctx->dp[k];
        const bool saved_tuned = ctx->dp_tuned;
        for (int i = 0; i < 7; ++i)
            if (!ctx->dp_tuned) ctx->dp[i] = ctx->def;
        ctx->dp_tuned = true;
        auto try_cfg = [&](const KCfg& c) {
            ctx->dp[k] = c;
            float ms = 0.f;
            if ((st = time_dp_kernel(ctx, k, 3, e0, e1, &ms)) != GS_OK) return;
            if (ms < best) {
                best = ms;
                best_cfg[k] = c;
            }
        };
        const bool staged_only = k >= 5 && split67_on(ctx);
        for (int fi = 0; fi < nf && st == GS_OK; ++fi) {
            if (staged_only && forms[fi] != 4) continue;
            if (forms[fi] == 4) {
                for (int ty = 2; ty <= kMaxTY && st == GS_OK; ++ty)
                    for (int depth = 1; depth <= 2 && st == GS_OK; ++depth) try_cfg(KCfg{4, ty, 0, depth});
                continue;
            }
            for (const auto& c : cand) {
                if (st != GS_OK) break;
                if (k == 6 && c[0] > kMaxTYFinal) continue;
                try_cfg(KCfg{forms[fi], c[0], c[1]});
            }
        }
        ctx->dp[k] = saved;
        ctx->dp_tuned = saved_tuned;
        stage_best[k] = best;
        total += best;
    }
    // stage pairs: every tile height x ring depth 1..3, then the automatic
    // choice between pairs and single stages by the summed kernel times of an
    // attempt
    KCfg best_pc[5] = {ctx->pc[0], ctx->pc[1], ctx->pc[2], ctx->pc[3], ctx->pc[4]};
    float pair_total = 0.f, rk4_pair_total = 0.f, rk4_single = 0.f;
    const bool tune_pairs = form_ok(ctx, 4) && (ctx->variant == 0 || ctx->variant == 4) && ctx->fuse != 0;
    for (int pi = 0; pi < 5 && tune_pairs && st == GS_OK; ++pi) {
        float best = 1e30f;
        const KCfg saved = ctx->pc[pi];
        for (int ty = 2; ty <= pair_max_ty(pair_mode(pi)) && st == GS_OK; ++ty)
            for (int depth = 1; depth <= kMaxDepth && st == GS_OK; ++depth) {
                ctx->pc[pi] = KCfg{5, ty, 0, depth};
                int used[5];
                gs_get_pair_depths_in_use(ctx, used);
                if (used[pi] < depth) break;  // shared memory holds no deeper ring
                float ms = 0.f;
                if ((st = time_pair_kernel(ctx, pi, 3, e0, e1, &ms)) != GS_OK) break;
                if (ms < best) {
                    best = ms;
                    best_pc[pi] = ctx->pc[pi];
                }
            }
        ctx->pc[pi] = saved;
        (pi < 3 ? pair_total : rk4_pair_total) += best;
    }
    // the single-stage RK4 step with the configuration the other integrators use
    if (tune_pairs && st == GS_OK) {
        const KCfg saved_def = ctx->def;
        ctx->def = best_cfg[1];
        const int saved_fuse = ctx->fuse;
        ctx->fuse = 0;
        float acc = 0.f;
        for (int r = 0; r < 4 && st == GS_OK; ++r) {
            init_fixed_ctrl(ctx, 0.0, 1e-3, 1 << 30);
            if ((st = upload_ctrl(ctx)) != GS_OK) break;
            cudaError_t e = cudaEventRecord(e0, ctx->stream);
            if (e == cudaSuccess) e = body_rk4(ctx, ctx->stream, 0, 0, false);
            if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                set_err(ctx, e, "autotune RK4 step");
                st = GS_ERR_CUDA;
            }
            if (r > 0) acc += ms;
        }
        rk4_single = acc / 3;
        ctx->fuse = saved_fuse;
        ctx->def = saved_def;
    }
    cudaStreamSynchronize(ctx->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GS_OK) return st;
    for (int k = 0; k < 7; ++k) ctx->dp[k] = best_cfg[k];
    ctx->dp_tuned = true;
    if (tune_pairs) {
        for (int pi = 0; pi < 5; ++pi) ctx->pc[pi] = best_pc[pi];
        ctx->fuse_auto = pair_total < total - stage_best[0];
        ctx->rk4_fuse_auto = rk4_pair_total < rk4_single;
    }
    // the other integrators use the configuration of the one-input stage
    ctx->def = best_cfg[1];
    drop_graphs(ctx);
    if (ty_out) *ty_out = ctx->def.ty;
    if (zc_out) *zc_out = ctx->def.zc;
    if (best_ms) *best_ms = total;  // sum of the best kernel times (k1 included)
    return GS_OK;
}

gs_status gs_time_stages(gs_ctx* ctx, int reps, double* ms) {
    if (!ctx || !ctx->state[0] || reps < 1 || !ms) return GS_ERR_INVALID;
    cudaEvent_t ev[8];
    for (int i = 0; i < 8; ++i) CK(cudaEventCreate(&ev[i]));
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    gs_status st = GS_OK;
    for (int r = 0; r < reps + 1 && st == GS_OK; ++r) {
        // fixed-step control block, parity 0: outputs go to the context's
        // second buffers only; the bound state is read, never written
        init_fixed_ctrl(ctx, 0.0, 1e-3, 1 << 30);
        if ((st = upload_ctrl(ctx)) != GS_OK) break;
        cudaError_t e = cudaEventRecord(ev[0], ctx->stream);
        if (e == cudaSuccess) e = launch_dopri5_k1(ctx, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], ctx->stream);
        for (int k = 2; k <= 7 && e == cudaSuccess; ++k) {
            e = launch_dopri5_stage(ctx, ctx->stream, k, 0, 0);
            if (e == cudaSuccess) e = cudaEventRecord(ev[k], ctx->stream);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[7]);
        for (int k = 0; k < 7 && e == cudaSuccess; ++k) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            if (r > 0) acc[k] += t;  // repetition 0 is a warm-up
        }
        if (e != cudaSuccess) {
            set_err(ctx, e, "gs_time_stages");
            st = GS_ERR_CUDA;
        }
    }
    for (int i = 0; i < 8; ++i) cudaEventDestroy(ev[i]);
    if (st != GS_OK) return st;
    for (int k = 0; k < 7; ++k) ms[k] = acc[k] / reps;
    return GS_OK;
}

gs_status gs_time_pairs(gs_ctx* ctx, int reps, double* ms) {
    if (!ctx || !ctx->state[0] || reps < 1 || !ms) return GS_ERR_INVALID;
    if (!form_ok(ctx, 4)) return GS_ERR_INVALID;
    cudaEvent_t ev[5];
    for (int i = 0; i < 5; ++i) CK(cudaEventCreate(&ev[i]));
    double acc[4] = {0, 0, 0, 0};
    gs_status st = GS_OK;
    for (int r = 0; r < reps + 1 && st == GS_OK; ++r) {
        init_fixed_ctrl(ctx, 0.0, 1e-3, 1 << 30);
        if ((st = upload_ctrl(ctx)) != GS_OK) break;
        cudaError_t e = cudaEventRecord(ev[0], ctx->stream);
        if (e == cudaSuccess) e = launch_dopri5_k1(ctx, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], ctx->stream);
        for (int pi = 0; pi < 3 && e == cudaSuccess; ++pi) {
            e = launch_dopri5_pair(ctx, ctx->stream, pi, 0, 0);
            if (e == cudaSuccess) e = cudaEventRecord(ev[pi + 2], ctx->stream);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[4]);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            if (r > 0) acc[k] += t;
        }
        if (e != cudaSuccess) {
            set_err(ctx, e, "gs_time_pairs");
            st = GS_ERR_CUDA;
        }
    }
    for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
    if (st != GS_OK) return st;
    for (int k = 0; k < 4; ++k) ms[k] = acc[k] / reps;
    return GS_OK;
}

const char* gs_last_error(const gs_ctx* ctx) { return ctx ? ctx->err : ""; }

}  // extern "C"
