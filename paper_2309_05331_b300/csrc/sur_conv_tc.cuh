// sur_conv_tc.cuh -- the surrogate's 32 -> 32 channel 3x3x3 periodic
// convolution on the 5th-generation tensor cores (tcgen05), BF16 x BF16 with
// FP32 accumulation in tensor memory (TMEM).
//
// Implicit GEMM per output z-plane of a tile: D[m][o] = sum_{tap, i}
// X[cell(m) + off(tap)][i] * Wfwd[tap][i][o], M = 128 cells (8 in x by 16 in
// y), N = 32 output channels, K = 27 taps x 32 channels = 54 MMAs of K = 16.
// A CTA owns a tile of 8 x 16 x 2 cells: two M = 128 accumulators of 32 FP32
// columns each in TMEM.
//
// Operands come straight from shared memory through matrix descriptors
// (K-major, no swizzle: 8-row x 16-byte core matrices; LBO = byte step
// between the two K halves of an MMA, SBO = byte step between 8-row groups).
//   A: the periodic input halo (10 x 18 x 4 cells) stored chunk-major,
//      [8-channel chunk][halo cell] x 16 bytes.  For any tap the 8 cells of
//      one x-run of the output tile are 8 consecutive halo cells, i.e. one
//      contiguous 128-byte core matrix; the 16 x-runs (y rows) are HX cells
//      apart (SBO = 160 bytes) and the next 8 channels are one chunk plane
//      further (LBO = 720 x 16 bytes).  So one descriptor per (tap, z, K half)
//      addresses the shifted activations in place: no im2col copy.
//   B: the packed weights re-laid once per CTA as [k-step][chunk][o] x 16
//      bytes (SBO = 128 bytes between 8 output rows, LBO = 512 bytes).
// One thread issues the 108 MMAs of a tile and commits them to an mbarrier;
// all 8 warps then read the accumulators (warp w: TMEM lanes 32 (w mod 4) ..,
// plane w / 4) and run the fused epilogue.  Two halo buffers and two
// accumulator sets (128 TMEM columns) pipeline the persistent tile loop: the
// halo of tile i+1 is copied (cp.async) while the MMAs of tile i run, and the
// epilogue of tile i overlaps the MMAs of tile i+1.  Every mbarrier wait has
// an iteration limit: on expiry the kernel counts the event in g_tc_timeouts,
// skips its remaining tiles, frees its TMEM and returns.
#pragma once

#include "sur_conv.cuh"

namespace sur {
namespace tc {

constexpr int TX = 8, TY = 16, TZ = 2;  // output tile; M = TX * TY = 128 per z-plane
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int HC = HX * HY * HZ;  // 720 halo cells
constexpr int CH = 32;            // channels in and out
constexpr int NCHUNK = CH / 8;    // 16-byte chunks per cell
constexpr int KS = 54;            // K steps of 16: 27 taps x 2 halves
constexpr int NTHREADS = 256;
constexpr uint32_t TMEM_COLS = 128;  // 2 sets x 2 planes of 128 x 32 FP32 accumulators
constexpr size_t W_BYTES = (size_t)KS * 2 * CH * 16;      // 55,296
constexpr size_t X_BYTES = (size_t)NCHUNK * HC * 16;      // 46,080 per halo buffer
constexpr size_t SMEM_BYTES = W_BYTES + 2 * X_BYTES + 32; // + 2 mbarriers and the TMEM address
constexpr long kMaxPolls = 1L << 22;                      // mbarrier wait limit (try_wait calls)

// kind::f16 instruction descriptor: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit
// 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CH >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

// Shared-memory matrix descriptor, no swizzle: start address, LBO and SBO in
// 16-byte units (14 bits each), descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_bf16_tmem(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
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
// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
    for (long i = 0; i < kMaxPolls; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
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
// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
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

// mbarrier waits that gave up (read by sur_conv_tc_status)
__device__ unsigned int g_tc_timeouts;

// Same contract as conv_fwd_kernel<32, 32, EPI> (sur_conv.cuh) for
// EPI in {BIAS_RELU_BF16, MASK_BF16, RAW_F32}; D % 2 == 0, H % 16 == 0,
// W % 8 == 0.  wp: the packed weights of sur_pack_weights.
// Periodic halo of tile (x0, y0, z0), chunk-major: chunk q of halo cell c at
// byte (q * HC + c) * 16; copied with cp.async (this thread's copies only).
__device__ __forceinline__ void halo_async(unsigned char* Xs, const __nv_bfloat16* __restrict__ x, int x0, int y0,
                                           int z0, int D, int H, int W) {
    for (int idx = threadIdx.x; idx < HC * NCHUNK; idx += NTHREADS) {
        const int q = idx / HC, c = idx - q * HC;
        const int hx = c % HX, rr = c / HX, hy = rr % HY, hz = rr / HY;
        // periodic wrap of a coordinate in [-1, n]
        int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
        gx += gx < 0 ? W : (gx >= W ? -W : 0);
        gy += gy < 0 ? H : (gy >= H ? -H : 0);
        gz += gz < 0 ? D : (gz >= D ? -D : 0);
        const size_t g = ((size_t)gx + (size_t)W * ((size_t)gy + (size_t)H * gz)) * CH + 8 * q;
        const uint32_t dst = smem_u32(Xs + (size_t)idx * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(x + g) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// The 108 MMAs of one tile: halo buffer at shared address xs_addr, weights at
// ws_addr, accumulators (plane p: columns p * 32 ..) at d_tmem.  Descriptor
// start addresses advance by adding 16-byte units to the low field: the sum
// stays inside shared memory (< 2^18 bytes), so it never carries out of the
// 14-bit field.
__device__ __forceinline__ void issue_tile_mmas(uint32_t xs_addr, uint32_t ws_addr, uint32_t d_tmem) {
    const uint64_t a_base = sdesc(xs_addr, HC * 16, HX * 16);
    const uint64_t b_base = sdesc(ws_addr, CH * 16, 8 * 16);
#pragma unroll 1
    for (int p = 0; p < TZ; ++p) {
        const uint64_t ap = a_base + (uint64_t)(p * HX * HY);
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            const int tap = ks >> 1, h = ks & 1;
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            const int c0 = (dx + 1) + HX * ((dy + 1) + HY * (dz + 1));  // halo cell of output (0, 0, 0)
            mma_bf16_tmem(d_tmem + (uint32_t)(p * CH), ap + (uint64_t)(c0 + 2 * h * HC), b_base + (uint64_t)(ks * 64),
                          ks > 0 ? 1u : 0u);
        }
    }
}

// Same contract as conv_fwd_kernel<32, 32, EPI> (sur_conv.cuh) for
// EPI in {BIAS_RELU_BF16, MASK_BF16, RAW_F32}; D % 2 == 0, H % 16 == 0,
// W % 8 == 0.  wp: the packed weights of sur_pack_weights.
template <int EPI>
__global__ void __launch_bounds__(NTHREADS, 1)
    conv_tc_kernel(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ wp,
                   const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask, void* out, int D, int H,
                   int W) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* Ws = smem;
    unsigned char* Xs[2] = {smem + W_BYTES, smem + W_BYTES + X_BYTES};
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + W_BYTES + 2 * X_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ws_addr = smem_u32(Ws);
    const uint32_t xs_addr[2] = {smem_u32(Xs[0]), smem_u32(Xs[1])};
    const uint32_t mbar_addr[2] = {smem_u32(mbar), smem_u32(mbar + 1)};

    // weights: packed row (ks, n) holds chunks q = 0, 1 (swizzled by n);
    // re-laid as [ks][q][n] so 8 output rows of a chunk form a core matrix
    for (int i = tid; i < KS * 2 * CH; i += NTHREADS) {
        const int ks = i / (2 * CH), rem = i - ks * 2 * CH, q = rem / CH, n = rem - q * CH;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned char*>(wp) +
                                                             wrow_off(ks, n, q, CH)));
        *reinterpret_cast<uint4*>(Ws + ((size_t)(ks * 2 + q) * CH + n) * 16) = v;
    }
    if (warp == 0) tmem_alloc(smem_u32(tslot), TMEM_COLS);
    if (tid == 0) {
        mbar_init(mbar_addr[0], 1);
        mbar_init(mbar_addr[1], 1);
    }
    const int ntx = W / TX, nty = H / TY, ntz = D / TZ;
    const int ntiles = ntx * nty * ntz;
    auto tile_origin = [&](int tile, int& x0, int& y0, int& z0) {
        const int tx = tile % ntx, r = tile / ntx, ty = r % nty, tz = r / nty;
        x0 = tx * TX;
        y0 = ty * TY;
        z0 = tz * TZ;
    };
    int x0, y0, z0;
    const int G = gridDim.x;
    if (blockIdx.x < ntiles) {
        tile_origin(blockIdx.x, x0, y0, z0);
        halo_async(Xs[0], x, x0, y0, z0, D, H, W);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;
    if (tid == 0 && blockIdx.x < ntiles) {
        issue_tile_mmas(xs_addr[0], ws_addr, tbase);
        mma_commit(mbar_addr[0]);
    }
    uint32_t phase[2] = {0u, 0u};
    // this thread's accumulator row: plane zz, cell (mx, my) of the tile
    const int zz = warp >> 2, m = 32 * (warp & 3) + lane, mx = m % TX, my = m / TX;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += G, ++it) {
        const int cur = it & 1, nxt = cur ^ 1;
        const int tile_n = tile + G;
        // halo of the next tile into the other buffer (its last reader, the
        // MMAs of tile i-1, completed before the previous epilogue)
        if (tile_n < ntiles) {
            int a, b, c;
            tile_origin(tile_n, a, b, c);
            halo_async(Xs[nxt], x, a, b, c, D, H, W);
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            fence_smem_to_async();
        }
        __syncthreads();  // next halo complete; the previous epilogue's TMEM reads done
        if (tid == 0 && tile_n < ntiles) {
            fence_after_sync();
            issue_tile_mmas(xs_addr[nxt], ws_addr, tbase + (uint32_t)(nxt * TZ * CH));
            mma_commit(mbar_addr[nxt]);
        }
        const bool ok = mbar_wait_bounded(mbar_addr[cur], phase[cur]);
        phase[cur] ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicAdd(&g_tc_timeouts, 1u);
            break;
        }
        fence_after_sync();
        tile_origin(tile, x0, y0, z0);
        float v[32];
        tmem_ld32(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(cur * TZ * CH + zz * CH), v);
        const size_t cell = (size_t)(x0 + mx) + (size_t)W * ((size_t)(y0 + my) + (size_t)H * (z0 + zz));
        if (EPI == EPI_BIAS_RELU_BF16 || (EPI == EPI_RAW_F32 && bias)) {
#pragma unroll
            for (int o = 0; o < 32; ++o) v[o] += __ldg(bias + o);
        }
        if (EPI == EPI_BIAS_RELU_BF16) {
#pragma unroll
            for (int o = 0; o < 32; ++o) v[o] = fmaxf(v[o], 0.f);
        }
        if (EPI == EPI_MASK_BF16) {
            const uint4* mp = reinterpret_cast<const uint4*>(mask + cell * CH);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const uint4 mv = __ldg(mp + qq);
                const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mv);
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (!(__bfloat162float(mb[e]) > 0.f)) v[8 * qq + e] = 0.f;
            }
        }
        if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_BF16) {
            uint4* po = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + cell * CH);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                uint4 w4;
                __nv_bfloat162* wb = reinterpret_cast<__nv_bfloat162*>(&w4);
#pragma unroll
                for (int e = 0; e < 4; ++e) wb[e] = __floats2bfloat162_rn(v[8 * qq + 2 * e], v[8 * qq + 2 * e + 1]);
                po[qq] = w4;
            }
        } else {
            float4* po = reinterpret_cast<float4*>(static_cast<float*>(out) + cell * CH);
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) po[qq] = make_float4(v[4 * qq], v[4 * qq + 1], v[4 * qq + 2], v[4 * qq + 3]);
        }
        fence_before_sync();  // ordered before the next MMAs into this set by the next __syncthreads
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tbase, TMEM_COLS);
}

}  // namespace tc
}  // namespace sur
