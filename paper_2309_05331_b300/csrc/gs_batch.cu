// gs_batch.cu -- error-controlled Dormand-Prince 5(4) for ensembles of
// independent Gray-Scott problems of uneven grid sizes and parameters.
//
// All instances live in one set of concatenated fields (instance i at element
// offset off_i).  Every instance has its own control block: time, step size,
// accept/reject, parity of its buffers, status.  Each Dormand-Prince stage is
// ONE persistent launch over all instances: CTAs take segments (instance,
// column of ty rows x 32 cells, run of zc planes) from an atomic counter, skip
// instances that have finished, and run the same segment code as the
// single-grid vectorised kernel (one cell per lane, so any nx works).  Stage 7
// folds each segment's error maximum into its instance's accumulator; a
// controller kernel (one thread per instance) then accepts or rejects every
// instance, picks its next step and sets the loop condition of the CUDA graph
// (WHILE any instance is still running).  With a ring depth d > 0 the
// segment code is the staged form (each thread copies its inputs d planes
// ahead into shared memory with cp.async), else the vectorised form.
//
// Stage pairs (gsb_set_pairs): stages 2+3, 4+5 and 6+7 each as one persistent
// launch over the segments, running the single-grid pair segment
// (gs_pair.cuh) with one cell per lane (any nx): k_i is recomputed on a
// one-cell ring instead of being stored and read back, so an attempt moves
// 18 field passes instead of 33; stages 6+7 fold each segment's error
// maximum into its instance's accumulator.
//
// Cache blocking by instance group: a whole batch's stage fields are many
// times the L2, but one instance's are small.  The instances are split into
// consecutive groups whose working set (state, stage fields) fits a budget
// of L2, and each attempt runs stages 2..7 group by group: a group's k2..k6
// are written and read again while they are still in L2, so HBM sees little
// more than each group's state, k1 and results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "gs_pair.cuh"
#include "gs_tile.cuh"
#include "gs_staged.cuh"
#include "gs_wide.cuh"
#include "gs_internal.h"
#include "host_util.h"

using namespace gsk;

namespace {

struct BInst {
    int nx, ny, nz;
    int vx;         // stage pairs: cells per lane (1, 2 or 4; the row alignment allows it)
    long long off;  // element offset in the concatenated fields
    double cx, cy, cz, Du, Dv, F, k;
};

struct BSeg {
    int inst, col, z0, z1;
};

constexpr int kBFields = 9;    // 0: second state buffer; 1..8: stage fields
// segment counters per group: stages 2..7, or the three stage pairs for each
// lane width (counter 0: the k1 stage)
constexpr int kStageCtrs = 9;
// segment lists: stage tiles, final-kernel tiles, pair tiles for 1, 2 and 4
// cells per lane
constexpr int kLists = 5;
// working set of a cell in units of the element size: state and second
// buffer, k1..k7, two components each
constexpr int kCellFields = 2 * (1 + kBFields);

// FP32: registers capped for 4 CTAs of 256 threads per SM (stage kernels,
// 64) or 3 (the final kernel, 85): the segment code prefetches a plane of
// raw inputs into registers and would otherwise halve its occupancy
template <typename T, int NK, int MODE>
__global__ void __launch_bounds__(MODE == MODE_STAGE ? 512 : 256,
                                  sizeof(T) == 4 ? (MODE == MODE_STAGE ? 2 : 3) : 1)
    gsb_stage_kernel(const BInst* __restrict__ insts, DevCtrl* ctrls, const BSeg* __restrict__ segs, int nseg,
                     unsigned int* counter, const StageArgs A, const int depth) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    unsigned char* R = smem_raw + (wide_smem_bytes<T, 1>(A.ty) + 15) / 16 * 16;  // staged form's ring
    __shared__ T red[32];
    __shared__ int s_seg;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    for (;;) {
        if (tid == 0) s_seg = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int sgi = s_seg;
        __syncthreads();  // every thread has read s_seg before it is replaced
        if (sgi >= nseg) break;
        const BSeg sg = segs[sgi];
        const DevCtrl* c = ctrls + sg.inst;
        if (c->done) continue;  // block-uniform: control blocks are read-only here
        const BInst in = insts[sg.inst];
        Geom<T> g;
        g.nx = in.nx;
        g.ny = in.ny;
        g.nz = in.nz;
        g.cx = (T)in.cx;
        g.cy = (T)in.cy;
        g.cz = (T)in.cz;
        g.Du = (T)in.Du;
        g.Dv = (T)in.Dv;
        g.F = (T)in.F;
        g.k = (T)in.k;
        const StagePtrs<T, NK> P = resolve_stage<T, NK, MODE>(A, c->parity, 0, in.off);
        const StageCoef<T, NK> C = stage_coef<T, NK>(A, c->dt_try, c->atol, c->rtol);
        const int ntx = (in.nx + 31) / 32;
        typename ErrBits<T>::U ebits = 0;
        if (depth > 0)
            staged_segment<T, NK, MODE, 1>(g, P, C, S, R, depth, A.ty, sg.col % ntx, sg.col / ntx, sg.z0, sg.z1,
                                           ebits);
        else
            wide_segment<T, NK, MODE, 1>(g, P, C, S, A.ty, sg.col % ntx, sg.col / ntx, sg.z0, sg.z1, ebits);
        const T emax = ErrBits<T>::value(ebits);
        if (MODE == MODE_DOPRI_FINAL) {
            const T bmax = block_nanmax(emax, red);
            if (tid == 0) atomic_max_nonneg(&ctrls[sg.inst].err_bits, (double)bmax);
        }
    }
}

// One Dormand-Prince stage pair of every running instance (MODE_PAIR_DOPRI23:
// stages 2+3 and the inverse error scale; MODE_PAIR_DOPRI45: stages 4+5 ->
// stage 6's fields;
// MODE_PAIR_DOPRI67: stages 6+7, y5, k7 and the instance's error maximum): CTAs take (instance, column of
// A.ty rows x 32 cells, run of planes) segments from the counter and run the
// pair segment with one cell per lane.
// Tile heights of the batch's pair segments: with one cell per lane, up to 7
// rows in a CTA compiled for two per SM (384 threads, <= 80 registers),
// 8..12 rows in one compiled for one per SM (544 threads: 17 warps, 5 on one
// SM sub-partition, so <= 96 registers; 12 rows measured faster than 11 rows
// in 16 warps at 128 registers).  12 is the most the pair segment's halo
// warp covers (2 lanes per row for ty + 4 rows).  Wider lanes (2 or 4 cells)
// run in the single grid's 12-warp CTA, one per SM, up to 7 rows.
constexpr int kBPairMaxTY = 12;
template <int VX, bool TALL>
__host__ __device__ constexpr int bpair_threads() {
    return 32 * ((TALL ? kBPairMaxTY : kPairMaxTY) + 5);
}
template <int VX, bool TALL>
__host__ __device__ constexpr int bpair_min_blocks() {
    return TALL ? 1 : pair_min_blocks<VX>();
}

template <typename T, int NK, int MODE, int VX, bool TALL>
__global__ void __launch_bounds__(bpair_threads<VX, TALL>(), (bpair_min_blocks<VX, TALL>()))
    gsb_pair_kernel(const BInst* __restrict__ insts, DevCtrl* ctrls, const BSeg* __restrict__ segs, int nseg,
                    unsigned int* counter, const StageArgs A, const int depth) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* SA = reinterpret_cast<T*>(smem_raw);
    T* SB = SA + 3 * (size_t)(A.ty + 4) * 2 * pair_pitch<T, VX>();
    unsigned char* SI = smem_raw + (pair_plane_bytes<T, VX>(A.ty) + 15) / 16 * 16;
    unsigned char* R = SI + pair_isc_bytes<T, MODE, VX>(A.ty);
    R += (128u - ((uint32_t)__cvta_generic_to_shared(R) & 127u)) & 127u;
    __shared__ T red[32];
    __shared__ int s_seg;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    for (;;) {
        if (tid == 0) s_seg = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int sgi = s_seg;
        __syncthreads();  // every thread has read s_seg before it is replaced
        if (sgi >= nseg) break;
        const BSeg sg = segs[sgi];
        const DevCtrl* c = ctrls + sg.inst;
        if (c->done) continue;  // block-uniform: control blocks are read-only here
        const BInst in = insts[sg.inst];
        Geom<T> g;
        g.nx = in.nx;
        g.ny = in.ny;
        g.nz = in.nz;
        g.cx = (T)in.cx;
        g.cy = (T)in.cy;
        g.cz = (T)in.cz;
        g.Du = (T)in.Du;
        g.Dv = (T)in.Dv;
        g.F = (T)in.F;
        g.k = (T)in.k;
        const StagePtrs<T, NK> P = resolve_stage<T, NK, MODE>(A, c->parity, 0, in.off);
        const PairCoef<T, NK> C = pair_coef<T, NK>(A, c->dt_try, c->atol, c->rtol);
        const int ntx = (in.nx + 32 * VX - 1) / (32 * VX);
        typename ErrBits<T>::U ebits = 0;
        pair_segment<T, NK, MODE, VX>(g, P, C, SA, SB, SI, R, depth, A.ty, sg.col % ntx, sg.col / ntx, sg.z0, sg.z1,
                                      ebits);
        if (MODE == MODE_PAIR_DOPRI67) {
            const T bmax = block_nanmax(ErrBits<T>::value(ebits), red);
            if (tid == 0) atomic_max_nonneg(&ctrls[sg.inst].err_bits, (double)bmax);
        }
    }
}

// One thread per instance: accept / reject, next step, stop.  Resets the
// stage segment counters (1 .. nctr-1) for the next attempt and sets the
// loop condition.
__global__ void __launch_bounds__(1024) gsb_controller_kernel(DevCtrl* ctrls, int n, unsigned int* counters, int nctr,
                                                              unsigned long long cond, int use_cond) {
    int active = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        DevCtrl* c = ctrls + i;
        if (!c->done) {
            const double E = __longlong_as_double((long long)c->err_bits);
            c->err_bits = 0ull;
            controller_update(c, E);
        }
        active |= c->done ? 0 : 1;
    }
    active = __syncthreads_or(active);
    for (int i = 1 + threadIdx.x; i < nctr; i += blockDim.x) counters[i] = 0u;
    if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, active ? 1u : 0u);
}

template <typename T>
__global__ void gsb_copy_back_kernel(const BInst* __restrict__ insts, const DevCtrl* ctrls, int n,
                                     const T* __restrict__ a0, const T* __restrict__ a1, T* __restrict__ b0,
                                     T* __restrict__ b1) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        if (ctrls[i].parity == 0) continue;
        const BInst in = insts[i];
        const long long N = (long long)in.nx * in.ny * in.nz;
        for (long long e = threadIdx.x; e < N; e += blockDim.x) {
            b0[in.off + e] = a0[in.off + e];
            b1[in.off + e] = a1[in.off + e];
        }
    }
}

}  // namespace

struct gsb_ctx {
    int count = 0;
    int prec = GS_FP32;
    size_t esz = 4;
    long long total = 0;
    std::vector<BInst> hinst;
    cudaStream_t stream = nullptr, cap = nullptr;
    int dev = 0, nsm = 0;
    void* state[2] = {nullptr, nullptr};
    unsigned char* scratch = nullptr;
    void* field[kBFields][2] = {};
    BInst* dinst = nullptr;
    DevCtrl* dctrl = nullptr;
    DevCtrl* hctrl = nullptr;  // pinned, count entries
    unsigned int* counters = nullptr;
    BSeg* dseg[kLists] = {};  // [0]: stage tiles, [1]: final-kernel tiles, [2 + c]: pair tiles, 2^c cells per lane
    int nseg[kLists] = {};
    int ty = 6, zc = 16;
    int depth = 0;                        // staged-form ring depth (0: vectorised form)
    int pairs = 0;                        // stage pairs (gsb_set_pairs)
    int pty = 7, pdepth = 2;              // pair tile height and ring depth (one cell per lane)
    int plane = 1, ptyw = kPairMaxTY;     // wider pair lanes where rows allow (gsb_set_pair_lanes), their tile height
    long long group_cells = 0;            // cells per group: -1 automatic (half the L2), 0 one group
    std::vector<int> gseg0[kLists], gsegn[kLists];  // per group: first segment and count in each list
    int ngroups = 1, nctr = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double* dlog = nullptr;  // accepted step sizes: log_cap per instance (gsb_set_step_log)
    long log_cap = 0;
    char err[512] = {0};
};

static void bset_err(gsb_ctx* c, cudaError_t e, const char* where) {
    if (c) snprintf(c->err, sizeof(c->err), "%s: %s", where, cudaGetErrorString(e));
}

#define BCK(call)                     \
    do {                              \
        cudaError_t e_ = (call);      \
        if (e_ != cudaSuccess) {      \
            bset_err(ctx, e_, #call); \
            return GS_ERR_CUDA;       \
        }                             \
    } while (0)

static void bdrop_graph(gsb_ctx* ctx) {
    if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    ctx->exec = nullptr;
    ctx->graph = nullptr;
}

static long long budget_cells(const gsb_ctx* ctx) {
    if (ctx->group_cells >= 0) return ctx->group_cells;
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->dev);
    return std::max<long long>(1, (long long)l2 / 2 / ((long long)kCellFields * (long long)ctx->esz));
}

// Cells per lane of an instance's stage pairs: lanes own 4 (FP32) or 2
// consecutive cells of a row when every row of the instance starts on that
// boundary (instances start 16-byte aligned, so nx a multiple of 4 or 2)
// and the row is long enough for the wider column (32 x 4 or 32 x 2 cells)
// not to leave most lanes idle: FP32 nx > 64 and a multiple of 4 -> 4
// cells, nx > 32 and even -> 2; FP64 (16-byte pairs) nx > 32 and even -> 2;
// otherwise (or with gsb_set_pair_lanes(ctx, 0, ...)) one cell per lane.
static int pair_lane_width(const gsb_ctx* ctx, int nx) {
    if (!ctx->plane) return 1;
    if (ctx->prec == GS_FP32 && nx > 64 && nx % 4 == 0) return 4;
    return (nx > 32 && nx % 2 == 0) ? 2 : 1;
}

// segment lists for rows-per-CTA ty (stages), min(ty, 6) (stage 7) and pty
// (stage pairs), and the instance groups (consecutive instances, at most
// budget_cells cells, at least one instance each)
static gs_status build_segments(gsb_ctx* ctx) {
    std::vector<int> first_inst;  // first instance of each group
    {
        const long long budget = budget_cells(ctx);
        long long acc = 0;
        for (int i = 0; i < ctx->count; ++i) {
            const BInst& in = ctx->hinst[i];
            const long long n = (long long)in.nx * in.ny * in.nz;
            if (i == 0 || (budget > 0 && acc + n > budget && acc > 0)) {
                first_inst.push_back(i);
                acc = 0;
            }
            acc += n;
        }
    }
    ctx->ngroups = (int)first_inst.size();
    for (int i = 0; i < ctx->count; ++i) ctx->hinst[i].vx = pair_lane_width(ctx, ctx->hinst[i].nx);
    for (int li = 0; li < kLists; ++li) {
        const int vx = li < 2 ? 1 : 1 << (li - 2);
        const int ty = li == 0 ? ctx->ty : (li == 1 ? std::min(ctx->ty, kMaxTYFinal) : (vx == 1 ? ctx->pty : ctx->ptyw));
        std::vector<BSeg> v;
        ctx->gseg0[li].assign(ctx->ngroups, 0);
        ctx->gsegn[li].assign(ctx->ngroups, 0);
        int g = 0;
        for (int i = 0; i < ctx->count; ++i) {
            if (g + 1 < ctx->ngroups && i == first_inst[g + 1]) ++g;
            if (i == first_inst[g]) ctx->gseg0[li][g] = (int)v.size();
            const BInst& in = ctx->hinst[i];
            if (li >= 2 && in.vx != vx) continue;  // pair lists: the instances of this lane width
            const int ncol = ((in.nx + 32 * vx - 1) / (32 * vx)) * ((in.ny + ty - 1) / ty);
            // z-chunk major: segments taken one after another cover the same
            // planes of neighbouring columns, so their halos meet in L2
            for (int z0 = 0; z0 < in.nz; z0 += ctx->zc)
                for (int col = 0; col < ncol; ++col) v.push_back(BSeg{i, col, z0, std::min(in.nz, z0 + ctx->zc)});
            ctx->gsegn[li][g] = (int)v.size() - ctx->gseg0[li][g];
        }
        if (ctx->dseg[li]) cudaFree(ctx->dseg[li]);
        ctx->dseg[li] = nullptr;
        ctx->nseg[li] = 0;
        if (v.empty()) continue;  // no instance of this lane width
        BCK(cudaMalloc(&ctx->dseg[li], sizeof(BSeg) * v.size()));
        BCK(cudaMemcpy(ctx->dseg[li], v.data(), sizeof(BSeg) * v.size(), cudaMemcpyHostToDevice));
        ctx->nseg[li] = (int)v.size();
    }
    const int nctr = 1 + kStageCtrs * ctx->ngroups;
    if (nctr != ctx->nctr) {
        if (ctx->counters) cudaFree(ctx->counters);
        ctx->counters = nullptr;
        ctx->nctr = 0;
        BCK(cudaMalloc(&ctx->counters, sizeof(unsigned int) * nctr));
        ctx->nctr = nctr;
    }
    BCK(cudaMemset(ctx->counters, 0, sizeof(unsigned int) * nctr));
    return GS_OK;
}

// launch over segments [seg0, seg0 + nseg) of the tile list of this mode,
// taken from the segment counter `counter`
template <typename T, int NK, int MODE>
static cudaError_t blaunch_t(gsb_ctx* ctx, cudaStream_t s, StageArgs A, int group, int counter) {
    const int li = MODE == MODE_STAGE ? 0 : 1;
    const int seg0 = group < 0 ? 0 : ctx->gseg0[li][group];
    const int nseg = group < 0 ? ctx->nseg[li] : ctx->gsegn[li][group];
    A.ty = li == 0 ? ctx->ty : std::min(ctx->ty, kMaxTYFinal);
    auto kern = gsb_stage_kernel<T, NK, MODE>;
    const size_t smem = ctx->depth > 0 ? staged_smem_bytes<T, NK, 1>(A.ty, ctx->depth) : wide_smem_bytes<T, 1>(A.ty);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * (A.ty + 2), smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const int grid = std::max(1, std::min(nseg, ctx->nsm * occ));
    kern<<<grid, dim3(32, A.ty + 2), smem, s>>>(ctx->dinst, ctx->dctrl, ctx->dseg[li] + seg0, nseg,
                                                ctx->counters + counter, A, ctx->depth);
    return cudaGetLastError();
}

template <int NK, int MODE>
static cudaError_t blaunch_nk(gsb_ctx* ctx, cudaStream_t s, const StageArgs& A, int g, int slot) {
    if (ctx->prec == GS_FP64) return blaunch_t<double, NK, MODE>(ctx, s, A, g, slot);
    return blaunch_t<float, NK, MODE>(ctx, s, A, g, slot);
}

static cudaError_t blaunch(gsb_ctx* ctx, cudaStream_t s, int nk, int mode, const StageArgs& A, int g, int slot) {
    if (mode == MODE_STAGE) {
        switch (nk) {
            case 0: return blaunch_nk<0, MODE_STAGE>(ctx, s, A, g, slot);
            case 1: return blaunch_nk<1, MODE_STAGE>(ctx, s, A, g, slot);
            case 2: return blaunch_nk<2, MODE_STAGE>(ctx, s, A, g, slot);
            case 3: return blaunch_nk<3, MODE_STAGE>(ctx, s, A, g, slot);
            case 4: return blaunch_nk<4, MODE_STAGE>(ctx, s, A, g, slot);
            case 5: return blaunch_nk<5, MODE_STAGE>(ctx, s, A, g, slot);
            default: return cudaErrorInvalidValue;
        }
    }
    if (mode == MODE_DOPRI_FINAL && nk == 5) return blaunch_nk<5, MODE_DOPRI_FINAL>(ctx, s, A, g, slot);
    return cudaErrorInvalidValue;
}

static Slot bfld(gsb_ctx* c, int f) { return slot_fixed(c->field[f][0], c->field[f][1]); }
static Slot bstate(gsb_ctx* c, int sel) {
    Slot s{};
    s.p[0][0] = c->state[0];
    s.p[0][1] = c->state[1];
    s.p[1][0] = c->field[0][0];
    s.p[1][1] = c->field[0][1];
    s.sel = sel;
    return s;
}
static Slot bpair(gsb_ctx* c, int fa, int fb, int sel) {
    Slot s{};
    s.p[0][0] = c->field[fa][0];
    s.p[0][1] = c->field[fa][1];
    s.p[1][0] = c->field[fb][0];
    s.p[1][1] = c->field[fb][1];
    s.sel = sel;
    return s;
}

// stage st (1 = k1, 2..7) of instance group g (k1: every instance, g < 0):
// same buffers and coefficients as the single grid
static cudaError_t blaunch_dopri5_stage(gsb_ctx* ctx, cudaStream_t s, int st, int g) {
    const int ctr = st == 1 ? 0 : 1 + kStageCtrs * g + (st - 2);
    const Slot k1 = bpair(ctx, 1, 2, SEL_CUR);
    const Slot k[7] = {k1, k1, bfld(ctx, 3), bfld(ctx, 4), bfld(ctx, 5), bfld(ctx, 6), bfld(ctx, 7)};
    static const double A2[1] = {dp5::A21};
    static const double A3[2] = {dp5::A31, dp5::A32};
    static const double A4[3] = {dp5::A41, dp5::A42, dp5::A43};
    static const double A5[4] = {dp5::A51, dp5::A52, dp5::A53, dp5::A54};
    static const double A6[5] = {dp5::A61, dp5::A62, dp5::A63, dp5::A64, dp5::A65};
    static const double* rows[5] = {A2, A3, A4, A5, A6};
    StageArgs A;
    memset(&A, 0, sizeof(A));
    A.u = bstate(ctx, SEL_CUR);
    if (st == 1) {
        A.out0 = k1;
        return blaunch(ctx, s, 0, MODE_STAGE, A, -1, 0);
    }
    if (st < 7) {
        const int nk = st - 1;
        for (int j = 0; j < nk; ++j) {
            A.kin[j] = k[j + 1];
            A.a[j] = rows[st - 2][j];
        }
        A.out0 = k[st];
        return blaunch(ctx, s, nk, MODE_STAGE, A, g, ctr);
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
    A.out0 = bstate(ctx, SEL_NEXT);
    A.out1 = bpair(ctx, 1, 2, SEL_NEXT);
    A.has_out1 = 1;
    return blaunch(ctx, s, 5, MODE_DOPRI_FINAL, A, g, ctr);
}

// one pair launch over group `group`'s instances of lane width VX (their
// own segment list), taken from the segment counter `counter`; nothing when
// the group has none
template <typename T, int NK, int MODE, int VX>
static cudaError_t bpair_launch_t(gsb_ctx* ctx, cudaStream_t s, StageArgs A, int group, int counter) {
    const int li = 2 + (VX == 4 ? 2 : VX - 1);
    const int seg0 = ctx->gseg0[li][group];
    const int nseg = ctx->gsegn[li][group];
    if (nseg == 0) return cudaSuccess;
    A.ty = VX == 1 ? ctx->pty : ctx->ptyw;
    auto kern = gsb_pair_kernel<T, NK, MODE, VX, false>;
    if constexpr (VX == 1)
        if (A.ty > kPairMaxTY) kern = gsb_pair_kernel<T, NK, MODE, VX, true>;
    int depth = std::max(1, std::min(ctx->pdepth, kMaxDepth));
    while (depth > 1 && pair_smem_bytes<T, NK, MODE, VX>(A.ty, depth) > kMaxSmemPerCta - 1024) --depth;
    const size_t smem = pair_smem_bytes<T, NK, MODE, VX>(A.ty, depth);
    if (smem > kMaxSmemPerCta - 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * (A.ty + 5), smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const int grid = std::max(1, std::min(nseg, ctx->nsm * occ));
    kern<<<grid, dim3(32, A.ty + 5), smem, s>>>(ctx->dinst, ctx->dctrl, ctx->dseg[li] + seg0, nseg,
                                                ctx->counters + counter, A, depth);
    return cudaGetLastError();
}
// pair pi of group g for every lane width (counters 3 per width apart)
template <int NK, int MODE>
static cudaError_t bpair_launch(gsb_ctx* ctx, cudaStream_t s, const StageArgs& A, int g, int pi) {
    const int ctr = 1 + kStageCtrs * g + pi;
    cudaError_t e = cudaSuccess;
    if (ctx->prec == GS_FP64) {
        e = bpair_launch_t<double, NK, MODE, 1>(ctx, s, A, g, ctr);
        if (e == cudaSuccess) e = bpair_launch_t<double, NK, MODE, 2>(ctx, s, A, g, ctr + 3);
        return e;
    }
    e = bpair_launch_t<float, NK, MODE, 1>(ctx, s, A, g, ctr);
    if (e == cudaSuccess) e = bpair_launch_t<float, NK, MODE, 2>(ctx, s, A, g, ctr + 3);
    if (e == cudaSuccess) e = bpair_launch_t<float, NK, MODE, 4>(ctx, s, A, g, ctr + 6);
    return e;
}

// Dormand-Prince stage pair pi (0: stages 2+3 and the inverse error scale ->
// field 8, 1: 4+5 -> Y6, P and the error terms in fields 5..7, 2: 6+7 from
// fields 5..8 -> y5, k7 and the error maxima) of instance group g: the
// buffers and coefficients of the single-grid pairs
static cudaError_t blaunch_dopri5_pair(gsb_ctx* ctx, cudaStream_t s, int pi, int g) {
    const Slot k1 = bpair(ctx, 1, 2, SEL_CUR);
    const Slot k[4] = {k1, k1, bfld(ctx, 3), bfld(ctx, 4)};  // k[i] = k_i
    StageArgs A;
    memset(&A, 0, sizeof(A));
    A.u = bstate(ctx, SEL_CUR);
    A.has_out1 = 1;
    if (pi == 0) {
        A.kin[0] = k[1];
        A.a[0] = dp5::A21;
        A.bk[0] = dp5::A31;
        A.bk[1] = dp5::A32;
        A.out0 = k[2];
        A.out1 = k[3];
        A.out2 = bfld(ctx, 8);  // inverse error scale
        return bpair_launch<1, MODE_PAIR_DOPRI23>(ctx, s, A, g, pi);
    }
    if (pi == 1) {
        static const double a4[3] = {dp5::A41, dp5::A42, dp5::A43};
        static const double a5[4] = {dp5::A51, dp5::A52, dp5::A53, dp5::A54};
        for (int j = 0; j < 3; ++j) {
            A.kin[j] = k[j + 1];
            A.a[j] = a4[j];
        }
        for (int j = 0; j < 4; ++j) A.bk[j] = a5[j];
        A.out0 = bfld(ctx, 5);  // Y6
        A.out1 = bfld(ctx, 6);  // P
        A.out2 = bfld(ctx, 7);  // error terms through k5
        return bpair_launch<3, MODE_PAIR_DOPRI45>(ctx, s, A, g, pi);
    }
    A.u = bfld(ctx, 5);
    A.kin[0] = bfld(ctx, 6);
    A.kin[1] = bfld(ctx, 7);
    A.kin[2] = bfld(ctx, 8);
    A.out0 = bstate(ctx, SEL_NEXT);       // y5
    A.out1 = bpair(ctx, 1, 2, SEL_NEXT);  // k7 = next k1
    return bpair_launch<3, MODE_PAIR_DOPRI67>(ctx, s, A, g, pi);
}

static cudaError_t bbody(gsb_ctx* ctx, cudaStream_t s, unsigned long long h, int use_cond, bool with_ctrl) {
    for (int g = 0; g < ctx->ngroups; ++g) {
        if (ctx->pairs) {
            for (int pi = 0; pi < 3; ++pi) {
                cudaError_t e = blaunch_dopri5_pair(ctx, s, pi, g);
                if (e != cudaSuccess) return e;
            }
            continue;
        }
        for (int st = 2; st <= 7; ++st) {
            cudaError_t e = blaunch_dopri5_stage(ctx, s, st, g);
            if (e != cudaSuccess) return e;
        }
    }
    if (!with_ctrl) return cudaSuccess;
    const int threads = std::min(1024, std::max(32, (ctx->count + 31) / 32 * 32));
    gsb_controller_kernel<<<1, threads, 0, s>>>(ctx->dctrl, ctx->count, ctx->counters, ctx->nctr, h, use_cond);
    return cudaGetLastError();
}

static gs_status bget_graph(gsb_ctx* ctx, cudaGraphExec_t* out) {
    if (ctx->exec) {
        *out = ctx->exec;
        return GS_OK;
    }
    cudaGraph_t g = nullptr, body = nullptr;
    cudaGraphConditionalHandle h;
    cudaError_t e = make_while_graph(&g, &h, &body);
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(ctx->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t eb = bbody(ctx, ctx->cap, (unsigned long long)h, 1, true);
        cudaGraph_t tmp = body;
        e = cudaStreamEndCapture(ctx->cap, &tmp);
        if (eb != cudaSuccess) e = eb;
    }
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        bset_err(ctx, e, "batched step graph");
        return GS_ERR_CUDA;
    }
    ctx->graph = g;
    ctx->exec = ex;
    *out = ex;
    return GS_OK;
}

extern "C" {

gs_status gsb_create(int count, const gsb_instance* inst, double L, double Du, double Dv, int prec, void* stream,
                     gsb_ctx** out) {
    if (!out) return GS_ERR_INVALID;
    *out = nullptr;
    if (count < 1 || count > 65536 || !inst || !(L > 0) || (prec != GS_FP32 && prec != GS_FP64))
        return GS_ERR_INVALID;
    for (int i = 0; i < count; ++i)
        if (inst[i].nx < 1 || inst[i].ny < 1 || inst[i].nz < 1 || inst[i].nx > 65535 || inst[i].ny > 65535 ||
            inst[i].nz > 65535)
            return GS_ERR_INVALID;
    gsb_ctx* ctx = new (std::nothrow) gsb_ctx();
    if (!ctx) return GS_ERR_NOMEM;
    ctx->count = count;
    ctx->prec = prec;
    ctx->esz = prec == GS_FP64 ? 8 : 4;
    ctx->stream = (cudaStream_t)stream;
    ctx->hinst.resize(count);
    long long off = 0;
    for (int i = 0; i < count; ++i) {
        BInst& b = ctx->hinst[i];
        b.nx = inst[i].nx;
        b.ny = inst[i].ny;
        b.nz = inst[i].nz;
        b.vx = 1;
        b.off = off;
        const double hx = L / b.nx, hy = L / b.ny, hz = L / b.nz;
        b.cx = 1.0 / (hx * hx);
        b.cy = 1.0 / (hy * hy);
        b.cz = 1.0 / (hz * hz);
        b.Du = Du;
        b.Dv = Dv;
        b.F = inst[i].F;
        b.k = inst[i].k;
        off += ((long long)b.nx * b.ny * b.nz + 3) / 4 * 4;  // instances start 16-byte aligned
    }
    ctx->total = off;
    gs_status st = GS_OK;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaGetDevice(&ctx->dev)) != cudaSuccess) break;
        if ((e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->dev)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking)) != cudaSuccess) break;
        const size_t fbytes = ((size_t)ctx->total * ctx->esz + 255) / 256 * 256;
        if ((e = cudaMalloc(&ctx->scratch, fbytes * 2 * kBFields)) != cudaSuccess) {
            st = GS_ERR_NOMEM;
            break;
        }
        for (int f = 0; f < kBFields; ++f)
            for (int c = 0; c < 2; ++c) ctx->field[f][c] = ctx->scratch + fbytes * (2 * f + c);
        if ((e = cudaMalloc(&ctx->dinst, sizeof(BInst) * count)) != cudaSuccess) break;
        if ((e = cudaMemcpy(ctx->dinst, ctx->hinst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            break;
        if ((e = cudaMalloc(&ctx->dctrl, sizeof(DevCtrl) * count)) != cudaSuccess) break;
        if ((e = cudaMemset(ctx->dctrl, 0, sizeof(DevCtrl) * count)) != cudaSuccess) break;
        if ((e = cudaMallocHost(&ctx->hctrl, sizeof(DevCtrl) * count)) != cudaSuccess) break;
    } while (0);
    if (e == cudaSuccess && st == GS_OK) st = build_segments(ctx);
    if (e != cudaSuccess || st != GS_OK) {
        if (st == GS_OK) st = (e == cudaErrorMemoryAllocation) ? GS_ERR_NOMEM : GS_ERR_CUDA;
        if (e != cudaSuccess) set_global_error(e, "gsb_create");
        gsb_destroy(ctx);
        return st;
    }
    *out = ctx;
    return GS_OK;
}

gs_status gsb_destroy(gsb_ctx* ctx) {
    if (!ctx) return GS_OK;
    bdrop_graph(ctx);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->dinst) cudaFree(ctx->dinst);
    if (ctx->dctrl) cudaFree(ctx->dctrl);
    if (ctx->hctrl) cudaFreeHost(ctx->hctrl);
    if (ctx->dlog) cudaFree(ctx->dlog);
    if (ctx->counters) cudaFree(ctx->counters);
    for (int i = 0; i < kLists; ++i)
        if (ctx->dseg[i]) cudaFree(ctx->dseg[i]);
    delete ctx;
    return GS_OK;
}

gs_status gsb_layout(const gsb_ctx* ctx, long long* offsets) {
    if (!ctx || !offsets) return GS_ERR_INVALID;
    for (int i = 0; i < ctx->count; ++i) offsets[i] = ctx->hinst[i].off;
    offsets[ctx->count] = ctx->total;
    return GS_OK;
}

gs_status gsb_bind_state(gsb_ctx* ctx, void* u, void* v) {
    if (!ctx || !u || !v || (((uintptr_t)u | (uintptr_t)v) & 15)) return GS_ERR_INVALID;
    if (ctx->state[0] != u || ctx->state[1] != v) bdrop_graph(ctx);
    ctx->state[0] = u;
    ctx->state[1] = v;
    return GS_OK;
}

gs_status gsb_set_tile(gsb_ctx* ctx, int ty, int zc) {
    if (!ctx || !(ty == 2 || ty == 4 || ty == 6 || ty == 8 || ty == 14) || zc < 1 || zc > 1024)
        return GS_ERR_INVALID;
    if (ty == ctx->ty && zc == ctx->zc) return GS_OK;
    bdrop_graph(ctx);
    ctx->ty = ty;
    ctx->zc = zc;
    return build_segments(ctx);
}

gs_status gsb_set_pairs(gsb_ctx* ctx, int on, int ty, int depth) {
    if (!ctx || on < 0 || on > 1 || ty < 1 || ty > kBPairMaxTY || depth < 1 || depth > kMaxDepth)
        return GS_ERR_INVALID;
    bdrop_graph(ctx);
    ctx->pairs = on;
    ctx->pdepth = depth;
    if (ty != ctx->pty) {
        ctx->pty = ty;
        return build_segments(ctx);
    }
    return GS_OK;
}

gs_status gsb_set_pair_lanes(gsb_ctx* ctx, int mode, int ty_wide) {
    if (!ctx || mode < 0 || mode > 1 || ty_wide < 1 || ty_wide > kPairMaxTY) return GS_ERR_INVALID;
    if (mode == ctx->plane && ty_wide == ctx->ptyw) return GS_OK;
    bdrop_graph(ctx);
    ctx->plane = mode;
    ctx->ptyw = ty_wide;
    return build_segments(ctx);
}

gs_status gsb_get_pair_lanes(const gsb_ctx* ctx, int* mode, int* ty_wide, int* counts) {
    if (!ctx) return GS_ERR_INVALID;
    if (mode) *mode = ctx->plane;
    if (ty_wide) *ty_wide = ctx->ptyw;
    if (counts) {
        counts[0] = counts[1] = counts[2] = 0;
        for (const BInst& in : ctx->hinst) ++counts[in.vx == 4 ? 2 : in.vx - 1];
    }
    return GS_OK;
}

gs_status gsb_get_pairs(const gsb_ctx* ctx, int* on, int* ty, int* depth) {
    if (!ctx) return GS_ERR_INVALID;
    if (on) *on = ctx->pairs;
    if (ty) *ty = ctx->pty;
    if (depth) *depth = ctx->pdepth;
    return GS_OK;
}

gs_status gsb_set_stage_depth(gsb_ctx* ctx, int depth) {
    if (!ctx || depth < 0 || depth > kMaxDepth) return GS_ERR_INVALID;
    if (depth == ctx->depth) return GS_OK;
    bdrop_graph(ctx);
    ctx->depth = depth;
    return GS_OK;
}

gs_status gsb_set_grouping(gsb_ctx* ctx, long long cells_per_group) {
    if (!ctx || cells_per_group < -1) return GS_ERR_INVALID;
    if (cells_per_group == ctx->group_cells) return GS_OK;
    bdrop_graph(ctx);
    ctx->group_cells = cells_per_group;
    return build_segments(ctx);
}

gs_status gsb_get_grouping(const gsb_ctx* ctx, long long* cells_per_group, int* ngroups) {
    if (!ctx) return GS_ERR_INVALID;
    if (cells_per_group) *cells_per_group = budget_cells(ctx);
    if (ngroups) *ngroups = ctx->ngroups;
    return GS_OK;
}

gs_status gsb_set_step_log(gsb_ctx* ctx, long capacity) {
    if (!ctx || capacity < 0) return GS_ERR_INVALID;
    if (ctx->dlog) {
        cudaFree(ctx->dlog);
        ctx->dlog = nullptr;
    }
    ctx->log_cap = 0;
    if (capacity == 0) return GS_OK;
    cudaError_t e = cudaMalloc(&ctx->dlog, sizeof(double) * (size_t)capacity * ctx->count);
    if (e != cudaSuccess) {
        ctx->dlog = nullptr;
        bset_err(ctx, e, "gsb_set_step_log");
        return e == cudaErrorMemoryAllocation ? GS_ERR_NOMEM : GS_ERR_CUDA;
    }
    ctx->log_cap = capacity;
    return GS_OK;
}

gs_status gsb_get_step_log(gsb_ctx* ctx, double* dts_host, long capacity, long* counts) {
    if (!ctx || !dts_host || !counts || capacity < 0) return GS_ERR_INVALID;
    if (!ctx->dlog || capacity > ctx->log_cap) return GS_ERR_INVALID;
    for (int i = 0; i < ctx->count; ++i) {
        const long n = (long)ctx->hctrl[i].n_acc;
        counts[i] = n;
        const long m = std::min(n, capacity);
        if (m > 0)
            BCK(cudaMemcpyAsync(dts_host + (size_t)i * capacity, ctx->dlog + (size_t)i * ctx->log_cap,
                                sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, ctx->stream));
    }
    BCK(cudaStreamSynchronize(ctx->stream));
    return GS_OK;
}

gs_status gsb_integrate_adaptive(gsb_ctx* ctx, double atol, double rtol, double* t, double t_end, double* dt,
                                 long max_accepted, long* n_acc, long* n_rej, int* status) {
    if (!ctx || !t || !dt || !ctx->state[0]) return GS_ERR_INVALID;
    if (!(atol >= 0) || !(rtol >= 0) || !(atol > 0 || rtol > 0) || std::isnan(t_end)) return GS_ERR_INVALID;
    for (int i = 0; i < ctx->count; ++i)
        if (!(dt[i] > 0)) return GS_ERR_INVALID;
    int active = 0;
    for (int i = 0; i < ctx->count; ++i) {
        DevCtrl* h = ctx->hctrl + i;
        memset(h, 0, sizeof(DevCtrl));
        h->mode = CTRL_ADAPTIVE;
        h->t = t[i];
        h->t0 = t[i];
        h->t_end = t_end;
        h->dt = dt[i];
        h->atol = atol;
        h->rtol = rtol;
        h->max_acc = max_accepted < 0 ? -1 : max_accepted;
        h->max_att = kMaxAttempts;
        if (ctx->dlog) {
            h->log_dt = ctx->dlog + (size_t)i * ctx->log_cap;
            h->log_cap = ctx->log_cap;
        }
        if (!(h->t < t_end) || max_accepted == 0) {
            h->done = 1;
            continue;
        }
        double ht = dt[i];
        if (h->t + ht >= t_end) {
            ht = t_end - h->t;
            h->last = 1;
        }
        if (!(ht > 0.0) || h->t + ht == h->t) {
            h->status = GS_ERR_STEP_UNDERFLOW;
            h->done = 1;
            continue;
        }
        h->dt_try = ht;
        ++active;
    }
    BCK(cudaMemcpyAsync(ctx->dctrl, ctx->hctrl, sizeof(DevCtrl) * ctx->count, cudaMemcpyHostToDevice, ctx->stream));
    if (active > 0) {
        BCK(cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned int) * ctx->nctr, ctx->stream));
        BCK(blaunch_dopri5_stage(ctx, ctx->stream, 1, -1));
        cudaGraphExec_t ex;
        gs_status st = bget_graph(ctx, &ex);
        if (st != GS_OK) return st;
        BCK(cudaGraphLaunch(ex, ctx->stream));
        if (ctx->prec == GS_FP64)
            gsb_copy_back_kernel<double><<<std::min(ctx->count, ctx->nsm * 4), 256, 0, ctx->stream>>>(
                ctx->dinst, ctx->dctrl, ctx->count, (const double*)ctx->field[0][0], (const double*)ctx->field[0][1],
                (double*)ctx->state[0], (double*)ctx->state[1]);
        else
            gsb_copy_back_kernel<float><<<std::min(ctx->count, ctx->nsm * 4), 256, 0, ctx->stream>>>(
                ctx->dinst, ctx->dctrl, ctx->count, (const float*)ctx->field[0][0], (const float*)ctx->field[0][1],
                (float*)ctx->state[0], (float*)ctx->state[1]);
        BCK(cudaGetLastError());
    }
    BCK(cudaMemcpyAsync(ctx->hctrl, ctx->dctrl, sizeof(DevCtrl) * ctx->count, cudaMemcpyDeviceToHost, ctx->stream));
    BCK(cudaStreamSynchronize(ctx->stream));
    gs_status first = GS_OK;
    for (int i = 0; i < ctx->count; ++i) {
        const DevCtrl* h = ctx->hctrl + i;
        t[i] = h->t;
        dt[i] = h->dt;
        if (n_acc) n_acc[i] = (long)h->n_acc;
        if (n_rej) n_rej[i] = (long)h->n_rej;
        if (status) status[i] = h->status;
        if (first == GS_OK && h->status != GS_OK) first = (gs_status)h->status;
    }
    return first;
}

// device time of one attempt round (k1 stage + stages 2..7 of every group)
// with the current tile and grouping, averaged over 2 runs after a warm-up
static gs_status time_round(gsb_ctx* ctx, cudaEvent_t e0, cudaEvent_t e1, float* out) {
    float acc = 0.f;
    for (int r = 0; r < 3; ++r) {
        BCK(cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned int) * ctx->nctr, ctx->stream));
        BCK(cudaEventRecord(e0, ctx->stream));
        cudaError_t e = blaunch_dopri5_stage(ctx, ctx->stream, 1, -1);
        if (e == cudaSuccess) e = bbody(ctx, ctx->stream, 0, 0, false);
        if (e != cudaSuccess) {
            bset_err(ctx, e, "gsb_autotune");
            return GS_ERR_CUDA;
        }
        BCK(cudaEventRecord(e1, ctx->stream));
        BCK(cudaEventSynchronize(e1));
        float ms = 0.f;
        BCK(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0) acc += ms;  // repetition 0 warms up
    }
    *out = acc / 2;
    return GS_OK;
}

gs_status gsb_autotune(gsb_ctx* ctx, int* ty_out, int* zc_out, double* best_ms) {
    if (!ctx || !ctx->state[0]) return GS_ERR_INVALID;
    // the timing round has every instance running; a real integration also
    // has sparse rounds (finished instances' segments are still walked), so
    // only z-chunks of 16 planes or more are candidates (measured on 512
    // uneven instances to t = 20, an earlier build: zc = 8 took 119 ms, zc =
    // 32 101 ms)
    static const int cand[][2] = {{4, 16}, {6, 16}, {6, 32}, {6, 64}, {8, 32}, {14, 16}, {14, 32}};
    // control blocks for timing: every instance running, parity 0, dt 1e-3
    for (int i = 0; i < ctx->count; ++i) {
        DevCtrl* h = ctx->hctrl + i;
        memset(h, 0, sizeof(DevCtrl));
        h->mode = CTRL_ADAPTIVE;
        h->dt = h->dt_try = 1e-3;
        h->atol = h->rtol = 1e-6;
        h->t_end = INFINITY;
        h->max_acc = -1;
        h->max_att = kMaxAttempts;
    }
    BCK(cudaMemcpyAsync(ctx->dctrl, ctx->hctrl, sizeof(DevCtrl) * ctx->count, cudaMemcpyHostToDevice, ctx->stream));
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    float best = 1e30f;
    int bty = ctx->ty, bzc = ctx->zc;
    gs_status st = GS_OK;
    // tiles of the segment code in use (the staged form copies one cell per
    // lane with 4- or 8-byte cp.async: on 512 uneven instances it took 129 ms
    // against 101 ms for the vectorised form, and a dense timing round does
    // not show it, so the depth is left to gsb_set_stage_depth)
    for (const auto& c : cand) {
        float ms = 0.f;
        if ((st = gsb_set_tile(ctx, c[0], c[1])) != GS_OK || (st = time_round(ctx, e0, e1, &ms)) != GS_OK) break;
        if (ms < best) {
            best = ms;
            bty = c[0];
            bzc = c[1];
        }
    }
    // instance grouping for the chosen tile: one group, or groups of a
    // quarter, half, one or two times the automatic (half-L2) budget (on the
    // 512-instance ensemble one group wins: 101 ms against 172-450 ms, the
    // per-group launches being too small to fill the GPU)
    long long bgroup = ctx->group_cells;
    if (st == GS_OK && (st = gsb_set_tile(ctx, bty, bzc)) == GS_OK) {
        const long long saved = ctx->group_cells;
        ctx->group_cells = -1;
        const long long autob = budget_cells(ctx);
        ctx->group_cells = saved;
        const long long gcand[5] = {0, autob / 4, autob / 2, autob, 2 * autob};
        best = 1e30f;
        for (long long gc : gcand) {
            float ms = 0.f;
            if ((st = gsb_set_grouping(ctx, gc)) != GS_OK || (st = time_round(ctx, e0, e1, &ms)) != GS_OK) break;
            if (ms < best) {
                best = ms;
                bgroup = gc;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GS_OK) return st;
    if ((st = gsb_set_tile(ctx, bty, bzc)) != GS_OK) return st;
    if ((st = gsb_set_grouping(ctx, bgroup)) != GS_OK) return st;
    if (ty_out) *ty_out = bty;
    if (zc_out) *zc_out = bzc;
    if (best_ms) *best_ms = best;
    return GS_OK;
}

// Tile choice by timing the integration itself: every candidate tile runs
// the caller's integration (same tolerance, interval and initial step) from
// the bound state, which is saved first and restored after each run and at
// the end.  A dense timing round (gsb_autotune) has every instance running;
// a real run of an uneven ensemble has instances finishing at different
// times, and the two rank tiles differently.
gs_status gsb_autotune_run(gsb_ctx* ctx, double atol, double rtol, double t0, double t_end, double dt0, int* ty_out,
                           int* zc_out, double* best_ms) {
    if (!ctx || !ctx->state[0] || !(t0 < t_end) || !(dt0 > 0) || !(atol >= 0) || !(rtol >= 0) || !(atol + rtol > 0))
        return GS_ERR_INVALID;
    // (pairs, tile height, z-chunk): the single-stage tiles, then the stage
    // pairs (one cell per lane) at two tile heights
    static const int cand[][3] = {{0, 4, 16}, {0, 6, 16}, {0, 6, 32}, {0, 6, 64}, {0, 8, 32}, {0, 14, 16},
                                  {0, 14, 32}, {1, 7, 32}, {1, 7, 64}, {1, 7, 128}, {1, 10, 64}, {1, 12, 64},
                                  {1, 12, 128}};
    const size_t bytes = ctx->esz * (size_t)ctx->total;
    void* save[2] = {nullptr, nullptr};
    for (int c = 0; c < 2; ++c) {
        if (cudaMalloc(&save[c], bytes) != cudaSuccess) {
            if (save[0]) cudaFree(save[0]);
            return GS_ERR_NOMEM;
        }
        if (cudaMemcpyAsync(save[c], ctx->state[c], bytes, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
            cudaFree(save[0]);
            if (save[1]) cudaFree(save[1]);
            return GS_ERR_CUDA;
        }
    }
    std::vector<double> t(ctx->count), dt(ctx->count);
    cudaEvent_t e0, e1;
    gs_status st = GS_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = GS_ERR_CUDA;
    float best = 1e30f;
    int bty = ctx->ty, bzc = ctx->zc, bpairs = ctx->pairs, bpty = ctx->pty;
    const int sty = ctx->ty;
    auto restore = [&]() -> gs_status {
        for (int c = 0; c < 2; ++c)
            if (cudaMemcpyAsync(ctx->state[c], save[c], bytes, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
                return GS_ERR_CUDA;
        return GS_OK;
    };
    for (const auto& c : cand) {
        if (st != GS_OK) break;
        if (c[0]) {
            if ((st = gsb_set_tile(ctx, sty, c[2])) != GS_OK) break;
            if ((st = gsb_set_pairs(ctx, 1, c[1], ctx->pdepth)) != GS_OK) break;
        } else {
            if ((st = gsb_set_pairs(ctx, 0, ctx->pty, ctx->pdepth)) != GS_OK) break;
            if ((st = gsb_set_tile(ctx, c[1], c[2])) != GS_OK) break;
        }
        for (int rep = 0; rep < 2 && st == GS_OK; ++rep) {  // the first run also builds the graph
            if ((st = restore()) != GS_OK) break;
            for (int i = 0; i < ctx->count; ++i) {
                t[i] = t0;
                dt[i] = dt0;
            }
            if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) st = GS_ERR_CUDA;
            const gs_status r = st == GS_OK ? gsb_integrate_adaptive(ctx, atol, rtol, t.data(), t_end, dt.data(), -1,
                                                                    nullptr, nullptr, nullptr)
                                            : st;
            if (r == GS_ERR_CUDA || r == GS_ERR_INVALID || r == GS_ERR_NOMEM) st = r;
            if (st == GS_OK && (cudaEventRecord(e1, ctx->stream) != cudaSuccess ||
                                cudaEventSynchronize(e1) != cudaSuccess))
                st = GS_ERR_CUDA;
            float ms = 0.f;
            if (st == GS_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = GS_ERR_CUDA;
            if (st == GS_OK && rep == 1 && ms < best) {
                best = ms;
                bpairs = c[0];
                if (c[0])
                    bpty = c[1];
                else
                    bty = c[1];
                bzc = c[2];
            }
        }
    }
    if (st == GS_OK) st = restore();
    if (st == GS_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = GS_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(save[0]);
    cudaFree(save[1]);
    if (st != GS_OK) return st;
    if ((st = gsb_set_tile(ctx, bty, bzc)) != GS_OK) return st;
    if ((st = gsb_set_pairs(ctx, bpairs, bpty, ctx->pdepth)) != GS_OK) return st;
    if (ty_out) *ty_out = bpairs ? bpty : bty;
    if (zc_out) *zc_out = bzc;
    if (best_ms) *best_ms = best;
    return GS_OK;
}

const char* gsb_last_error(const gsb_ctx* ctx) { return ctx ? ctx->err : ""; }

}  // extern "C"
