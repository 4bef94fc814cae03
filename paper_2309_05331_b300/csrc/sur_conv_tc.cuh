// sur_conv_tc.cuh -- the surrogate's 32 -> 32 channel 3x3x3 periodic
// convolution on the 5th-generation tensor cores (tcgen05), BF16 x BF16 with
// FP32 accumulation in tensor memory (TMEM).
//
// Implicit GEMM, out[c][o] = sum_{tap, i} x[c + off(tap)][i] W[tap][i][o].
// A CTA owns an output tile of 8 (x) x 16 (y) x 4 (z) cells: M = 128 cells
// per z-plane.  The z-taps are stacked along N: for input plane q of the
// tile's halo and one (dy, dx) tap pair, ONE MMA multiplies the shifted
// input rows (M = 128, K = 16 channels) by [W(dz=+1); W(dz=0); W(dz=-1)]
// (N = 96) and lands the three products in the accumulators of output planes
// q-2, q-1 and q at once: the accumulator of output plane p occupies TMEM
// columns 32 (p + 2) .. 32 (p + 2) + 31, so an MMA writing columns
// 32 q .. 32 q + 95 adds W(+1) x into plane q-2, W(0) x into q-1 and
// W(-1) x into q.  Planes -2, -1, 4 and 5 of that range are sinks, never
// read.  An N = 32 MMA costs about as much as an N = 96 one on these tensor
// cores (both are bound by reading the 4 KB A operand), so stacking triples
// the useful work per MMA.  The first contribution to a plane's accumulator
// (input plane q, first (dy, dx, K half)) is split into an accumulating
// N = 64 MMA for planes q-2, q-1 and an overwriting N = 32 MMA for plane q,
// so no accumulator needs zeroing.  Per tile: 6 input planes x (18 + 1)
// = 114 MMAs.
//
// Operands come straight from shared memory through matrix descriptors
// (K-major, no swizzle: 8-row x 16-byte core matrices; LBO = byte step
// between the two K halves of an MMA, SBO = byte step between 8-row groups).
//   A: the periodic input halo (10 x 18 x 6 cells) stored chunk-major,
//      [8-channel chunk][halo cell] x 16 bytes.  For any tap the 8 cells of
//      one x-run of the output tile are 8 consecutive halo cells, i.e. one
//      contiguous 128-byte core matrix; the 16 x-runs (y rows) are HX cells
//      apart (SBO = 160 bytes) and the next 8 channels are one chunk plane
//      further (LBO = 1080 x 16 bytes): one descriptor per (plane, tap pair,
//      K half) addresses the shifted activations in place, no im2col copy.
//   B: the packed weights re-laid once per CTA as [dy, dx][K half][chunk]
//      [96 stacked output rows] x 16 bytes (SBO 128, LBO 1536 bytes).
//
// The 8-channel layers use the same kernel.  CIN = 8: a tap carries one
// 16-byte chunk, so an MMA (K = 16) pairs two (dy, dx) taps of the same input
// plane, the second core matrix LBO bytes after the first (the two taps'
// cell distance); 5 pairs cover the 9 taps (the tenth weight block is zero).
// COUT = 8: a plane's accumulator is 16 columns wide (8 zero weight rows),
// so the stacked MMA has N = 48 and the first-touch split N = 32 + 16.
//
// Warp-specialised persistent pipeline (9 warps): warp 8 allocates TMEM and
// issues each tile's MMAs from one thread; warps 0-7 copy halos (cp.async)
// and run the fused epilogue (warp w reads TMEM lanes 32 (w mod 4) .. of
// planes 2 (w / 4), 2 (w / 4) + 1).  Two halo buffers and two accumulator
// sets (2 x 256 TMEM columns) flow between them through mbarriers: halo full
// (256 loader arrivals) / halo empty (MMA commit), accumulators full (MMA
// commit) / empty (8 epilogue warps).  Once the MMAs of tile i complete, the
// loaders publish the halo of tile i+1 (copied meanwhile) and start copying
// that of tile i+2 into the buffer tile i used, then run the epilogue of
// tile i: the MMAs of tile i+1 and the copies for tile i+2 both run while
// the epilogue of tile i does, and the MMA warp never joins a block barrier.
// Every mbarrier wait has an iteration limit and also watches a shared abort
// flag: on expiry the kernel sets the caller's timeout word (host-mapped
// memory the host reads after the launch, so the call that owns the launch
// reports an error instead of a result), all roles leave their loops, and
// the TMEM is freed.
#pragma once

#include "sur_conv.cuh"

namespace sur {
namespace tc {

constexpr int TX = 8, TY = 16, TZ = 4;  // output tile; M = TX * TY = 128 per z-plane
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int HC = HX * HY * HZ;  // 1080 halo cells
constexpr int NTHREADS = 288;     // 8 loader / epilogue warps + 1 MMA warp
constexpr int NLOAD = 256;        // loader / epilogue threads
constexpr int NBUF = 2;           // halo buffers
constexpr long kMaxPolls = 1L << 22;  // mbarrier wait limit (try_wait calls)

// Shapes of one (CIN, COUT) instance; CIN, COUT in {8, 32} (padded counts).
template <int CIN, int COUT>
struct Cfg {
    static constexpr int NCI = CIN / 8;                   // 16-byte chunks per input cell
    static constexpr int CW = COUT == 32 ? 32 : 16;       // accumulator columns per plane
    static constexpr int NSTK = 3 * CW;                   // stacked B rows: W(dz=+1), W(0), W(-1)
    static constexpr int KG = CIN == 32 ? 18 : 5;         // K groups (MMAs) per input plane
    static constexpr int SET_COLS = (TZ + 4) * CW;        // planes -2 .. TZ+1
    static constexpr uint32_t TMEM_COLS = 2 * SET_COLS;   // two accumulator sets (512 or 256)
    static constexpr size_t W_BYTES = (size_t)KG * 2 * NSTK * 16;
    static constexpr size_t X_BYTES = (size_t)NCI * HC * 16;
    static constexpr size_t SMEM_BYTES = W_BYTES + NBUF * X_BYTES + 128;  // + mbarriers, TMEM address, abort flag
};

// kind::f16 instruction descriptor: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit
// 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_m128(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: start address, LBO and SBO in
// 16-byte units (14 bits each), descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_bf16_tmem(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor cores' reads
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity to complete; gives up
// (false) after kMaxPolls tries or once *abort is set, and then sets *abort;
// the first thread of the CTA to give up also sets the launch's timeout
// word (*timeouts = 1; a plain store: the word may live in host memory)
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, volatile int* abort,
                                                  unsigned int* timeouts) {
    for (long i = 0; i < kMaxPolls; ++i) {
        if (mbar_try_wait(mbar, parity)) return true;
        if ((i & 63) == 63 && *abort) return false;
    }
    if (atomicExch((int*)abort, 1) == 0) {
        *reinterpret_cast<volatile unsigned int*>(timeouts) = 1u;
        __threadfence_system();
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot_saddr, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot_saddr), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Periodic halo of the tile at (x0, y0, z0), chunk-major: chunk q of halo
// cell c at byte (q * HC + c) * 16; copied with cp.async (this thread's
// copies only).  NCI chunks (CIN = 8 NCI channels) per cell.  Consecutive
// threads take consecutive chunks of a cell, then of the next cell in x, so
// a warp reads whole cells (contiguous runs of x) and every 32-byte sector
// it touches is used whole.
template <int NCI>
__device__ __forceinline__ void halo_async(unsigned char* Xs, const __nv_bfloat16* __restrict__ x, int x0, int y0,
                                           int z0, int D, int H, int W) {
    for (int idx = threadIdx.x; idx < HC * NCI; idx += NLOAD) {
        const int q = idx % NCI, c = idx / NCI;
        const int hx = c % HX, rr = c / HX, hy = rr % HY, hz = rr / HY;
        // periodic wrap of a coordinate in [-1, n]
        int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
        gx += gx < 0 ? W : (gx >= W ? -W : 0);
        gy += gy < 0 ? H : (gy >= H ? -H : 0);
        gz += gz < 0 ? D : (gz >= D ? -D : 0);
        const size_t g = ((size_t)gx + (size_t)W * ((size_t)gy + (size_t)H * gz)) * (8 * NCI) + 8 * q;
        const uint32_t dst = smem_u32(Xs + (size_t)(q * HC + c) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(x + g) : "memory");
    }
}

// The MMAs of one tile: halo buffer at shared address xs_addr, stacked
// weights at ws_addr, accumulator set at d_tmem.  Descriptor start addresses
// advance by adding 16-byte units to the low field: the sum stays inside
// shared memory (< 2^18 bytes), so it never carries out of the 14-bit field.
// K group g of an input plane: CIN = 32: tap pair r = g / 2, channel half
// h = g % 2 (second core matrix one chunk plane further); CIN = 8: taps 2g
// and 2g+1 (second core matrix at the second tap's cell, or the first one
// again with zero weights for g = 4).
template <int CIN, int COUT>
__device__ __forceinline__ void issue_tile_mmas(uint32_t xs_addr, uint32_t ws_addr, uint32_t d_tmem) {
    using C = Cfg<CIN, COUT>;
    constexpr int CW = C::CW, NSTK = C::NSTK;
    const uint64_t b_base = sdesc(ws_addr, NSTK * 16, 8 * 16);
    constexpr uint32_t IDS = idesc_m128(NSTK), ID2 = idesc_m128(2 * CW), ID1 = idesc_m128(CW);
    auto cell0 = [](int r) { return (r % 3) + HX * (r / 3); };  // (dx+1) + HX (dy+1)
#pragma unroll 1
    for (int q = 0; q < HZ; ++q) {
        const uint32_t d = d_tmem + (uint32_t)(q * CW);  // planes q-2, q-1, q
#pragma unroll
        for (int g = 0; g < C::KG; ++g) {
            uint64_t ad;
            if (CIN == 32) {
                const int r = g >> 1, h = g & 1;
                ad = sdesc(xs_addr, HC * 16, HX * 16) + (uint64_t)(cell0(r) + HX * HY * q + 2 * h * HC);
            } else {
                const int ra = 2 * g, rb = 2 * g + 1;
                const uint32_t lbo = rb < 9 ? (uint32_t)((cell0(rb) - cell0(ra)) * 16) : 0u;
                ad = sdesc(xs_addr, lbo, HX * 16) + (uint64_t)(cell0(ra) + HX * HY * q);
            }
            const uint64_t bd = b_base + (uint64_t)(g * 2 * NSTK);
            if (g == 0) {
                // first contribution to plane q: accumulate into q-2, q-1, overwrite q
                mma_bf16_tmem(d, ad, bd, ID2, 1u);
                mma_bf16_tmem(d + 2 * CW, ad, bd + (uint64_t)(2 * CW), ID1, 0u);
            } else {
                mma_bf16_tmem(d, ad, bd, IDS, 1u);
            }
        }
    }
}

// Same contract as conv_fwd_kernel<CIN, COUT, EPI> (sur_conv.cuh); D % 4 == 0,
// H % 16 == 0, W % 8 == 0.  wp: the packed weights of sur_pack_weights.
// timeouts: set to 1 if a wait gave up (the output is then invalid).
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(NTHREADS, 1)
    conv_tc_kernel(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ wp,
                   const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask, void* out, int out_ch,
                   int D, int H, int W, unsigned int* timeouts) {
    using C = Cfg<CIN, COUT>;
    constexpr int CW = C::CW, NSTK = C::NSTK, SET_COLS = C::SET_COLS;
    constexpr size_t W_BYTES = C::W_BYTES, X_BYTES = C::X_BYTES;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* Ws = smem;
    unsigned char* Xs[NBUF];
    for (int b = 0; b < NBUF; ++b) Xs[b] = smem + W_BYTES + b * X_BYTES;
    // mbarriers: halo full [0, 1], halo empty [2, 3], accumulators full [4, 5], empty [6, 7]
    constexpr int HF = 0, HE = NBUF, AF = 2 * NBUF, AE = 2 * NBUF + 2;
    uint64_t* mb = reinterpret_cast<uint64_t*>(smem + W_BYTES + NBUF * X_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mb + AE + 2);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ws_addr = smem_u32(Ws);
    auto bar = [&](int k) -> uint32_t { return smem_u32(mb + k); };

    // stacked weights: B row n' = CW j + o of K group g, core-matrix column k
    // holds W(dz = 1 - j, tap of (g, k))[input chunk of (g, k)][o] (zero for
    // o >= COUT or a missing tap).  Packed rows: CIN = 32, row (ks = 2 tap +
    // h, o) holds chunks q = 0, 1 of channels 16 h + 8 q ..; CIN = 8, row (ks,
    // o) holds chunk q = tap of taps 2 ks, 2 ks + 1.  Chunks are swizzled by o.
    for (int i = tid; i < C::KG * 2 * NSTK; i += NTHREADS) {
        const int n = i % NSTK, gk = i / NSTK, k = gk & 1, g = gk >> 1;
        const int j = n / CW, o = n - j * CW, dz = 1 - j;
        int r, ks, q;
        if (CIN == 32) {
            r = g >> 1;
            ks = 2 * ((dz + 1) * 9 + r) + (g & 1);
            q = k;
        } else {
            r = 2 * g + k;
            const int tap = (dz + 1) * 9 + r;
            ks = tap >> 1;
            q = tap & 1;
        }
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (o < COUT && r < 9)
            v = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned char*>(wp) +
                                                     wrow_off(ks, o, q, COUT)));
        *reinterpret_cast<uint4*>(Ws + (size_t)i * 16) = v;
    }
    if (warp == 8) tmem_alloc(smem_u32(tslot), C::TMEM_COLS);
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(bar(HF + b), NLOAD);  // halo full: every loader thread
            mbar_init(bar(HE + b), 1);      // halo empty: MMA commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar(AF + b), 1);  // accumulators full: MMA commit
            mbar_init(bar(AE + b), 8);  // accumulators empty: one lane per epilogue warp
        }
        *abort = 0;
    }
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;

    const int ntx = W / TX, nty = H / TY, ntz = D / TZ;
    const int ntiles = ntx * nty * ntz;
    const int G = gridDim.x;
    const int nmine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / G + 1 : 0;  // tiles of this CTA
    auto tile_origin = [&](int i, int& x0, int& y0, int& z0) {
        const int tile = blockIdx.x + i * G;
        const int tx = tile % ntx, r = tile / ntx, ty = r % nty, tz = r / nty;
        x0 = tx * TX;
        y0 = ty * TY;
        z0 = tz * TZ;
    };

    if (warp == 8) {
        // MMA issuer: tile i reads halo buffer i % 2 into accumulator set i % 2
        // (the k-th use of a barrier waits for parity k & 1)
        if (lane == 0) {
            for (int i = 0; i < nmine; ++i) {
                const int b = i & 1;
                if (!mbar_wait_bounded(bar(HF + b), (uint32_t)((i >> 1) & 1), abort, timeouts)) break;
                if (i >= 2 && !mbar_wait_bounded(bar(AE + b), (uint32_t)(((i >> 1) - 1) & 1), abort, timeouts)) break;
                fence_after_sync();
                issue_tile_mmas<CIN, COUT>(smem_u32(Xs[b]), ws_addr, tbase + (uint32_t)(b * SET_COLS));
                mma_commit(bar(AF + b));  // accumulators full
                mma_commit(bar(HE + b));  // halo buffer free
            }
        }
        __syncwarp();
    } else {
        // loaders / epilogue
        auto load = [&](int i) {
            int a, b, c;
            tile_origin(i, a, b, c);
            halo_async<C::NCI>(Xs[i & 1], x, a, b, c, D, H, W);
        };
        auto publish = [&](int i) {  // this thread's copies of tile i are in shared memory
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            fence_smem_to_async();
            mbar_arrive(bar(HF + (i & 1)));
        };
        // halo i + 1 is copied while tile i's MMAs and epilogue run: it is
        // issued right after tile i - 1's MMAs complete (its buffer was last
        // read by them) and published right after tile i's MMAs complete,
        // before tile i's epilogue, so the MMAs of tile i + 1 also run while
        // the epilogue of tile i does
        if (nmine > 0) {
            load(0);
            publish(0);
        }
        if (nmine > 1) load(1);  // buffer 1: first use
        const int m = 32 * (warp & 3) + lane, mx = m % TX, my = m / TX;
        // the bias in registers for the whole launch (per-plane loads of it
        // would queue behind the halo copies)
        constexpr bool HAS_BIAS = EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_BIAS_F32 || EPI == EPI_RAW_F32;
        float bv[COUT];
#pragma unroll
        for (int o = 0; o < COUT; ++o) bv[o] = (HAS_BIAS && bias) ? __ldg(bias + o) : 0.f;
        for (int i = 0; i < nmine; ++i) {
            const int s = i & 1;
            if (!mbar_wait_bounded(bar(AF + s), (uint32_t)((i >> 1) & 1), abort, timeouts)) break;
            fence_after_sync();
            if (i + 1 < nmine) publish(i + 1);
            if (i + 2 < nmine) {
                // buffer s was last read by the MMAs of tile i (complete)
                if (!mbar_wait_bounded(bar(HE + s), (uint32_t)((((i + 2) >> 1) - 1) & 1), abort, timeouts)) break;
                load(i + 2);
            }
            int x0, y0, z0;
            tile_origin(i, x0, y0, z0);
#pragma unroll 1
            for (int pp = 0; pp < 2; ++pp) {
                const int p = 2 * (warp >> 2) + pp;  // output plane of the tile
                float v[CW];
                const uint32_t ta =
                    tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(s * SET_COLS + (p + 2) * CW);
                if (CW == 32)
                    tmem_ld32(ta, v);
                else
                    tmem_ld16(ta, v);
                if (pp == 1) {
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar(AE + s));  // this warp's accumulator rows are read
                }
                const size_t cell = (size_t)(x0 + mx) + (size_t)W * ((size_t)(y0 + my) + (size_t)H * (z0 + p));
                if (HAS_BIAS) {
#pragma unroll
                    for (int o = 0; o < COUT; ++o) v[o] += bv[o];
                }
                if (EPI == EPI_BIAS_RELU_BF16) {
#pragma unroll
                    for (int o = 0; o < COUT; ++o) v[o] = fmaxf(v[o], 0.f);
                }
                if (EPI == EPI_MASK_BF16) {
                    const uint4* mp = reinterpret_cast<const uint4*>(mask + cell * COUT);
#pragma unroll
                    for (int qq = 0; qq < COUT / 8; ++qq) {
                        const uint4 mv = __ldg(mp + qq);
                        const __nv_bfloat16* mbf = reinterpret_cast<const __nv_bfloat16*>(&mv);
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (!(__bfloat162float(mbf[e]) > 0.f)) v[8 * qq + e] = 0.f;
                    }
                }
                if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_BF16) {
                    uint4* po = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + cell * COUT);
#pragma unroll
                    for (int qq = 0; qq < COUT / 8; ++qq) {
                        uint4 w4;
                        __nv_bfloat162* wb = reinterpret_cast<__nv_bfloat162*>(&w4);
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            wb[e] = __floats2bfloat162_rn(v[8 * qq + 2 * e], v[8 * qq + 2 * e + 1]);
                        po[qq] = w4;
                    }
                } else if (EPI == EPI_BIAS_F32) {
                    float* po = static_cast<float*>(out) + cell * out_ch;
#pragma unroll
                    for (int o = 0; o < COUT; ++o)
                        if (o < out_ch) po[o] = v[o];
                } else {
                    float4* po = reinterpret_cast<float4*>(static_cast<float*>(out) + cell * COUT);
#pragma unroll
                    for (int qq = 0; qq < COUT / 4; ++qq)
                        po[qq] = make_float4(v[4 * qq], v[4 * qq + 1], v[4 * qq + 2], v[4 * qq + 3]);
                }
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 8) tmem_dealloc(tbase, C::TMEM_COLS);
}

}  // namespace tc
}  // namespace sur
