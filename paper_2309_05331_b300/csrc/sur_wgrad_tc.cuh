// sur_wgrad_tc.cuh -- weight gradient of the surrogate's 32 -> 32 channel
// convolution on the tcgen05 tensor cores:
//   dW[tap][i][o] = sum over cells c of x[c + off(tap)][i] dy[c][o].
//
// The weight rows (i, 32 of them) are too few for an M = 128 MMA, so each
// MMA also spans four z-shifts: with the input halo of a one-plane tile
// stored chunk-major over exactly 4 z-planes ([8-channel chunk q][z-plane
// z'][y][x] x 16 bytes, one chunk plane = 4 z-planes of Z = 10 x 18 cells),
// the 16 row groups (q, z') of 8 channels sit at the uniform byte step
// (4 q + z') Z 16, so ONE descriptor addresses A[(q, z', e)][cell] =
// x[cell + (dx, dy, z' - 1)][8 q + e] for all 32 channels and z-shifts
// -1, 0, +1 (and +2, a discarded row block).  A is MN-major (8 channels of a
// cell contiguous, consecutive cells of an x-run 16 bytes apart: a 128-byte
// core matrix), K = 16 cells = two x-runs of the tile (LBO = one halo row).
// B = dy[cell][o] of the tile, MN-major too ([chunk][cell] x 16 bytes).  So
// per (dy, dx) tap pair and K step one M = 128, N = 32 MMA accumulates dW for
// three dz-taps into the pair's TMEM accumulator (columns 32 (3 (dy+1) +
// (dx+1)) ..): 9 x 8 = 72 MMAs per 8 x 16 cell tile, accumulating over all
// of a CTA's tiles (288 TMEM columns).  The CTA finally reads its
// accumulators and writes its partial dW, which wgrad_reduce_kernel sums.
//
// Pipeline: the conv kernel's warp split (warp 8 issues MMAs, warps 0-7 copy
// tiles with cp.async), two tile buffers handed over by mbarriers with
// bounded waits; a last commit tells the epilogue warps that every MMA is
// done.
#pragma once

#include "sur_conv_tc.cuh"

namespace sur {
namespace wtc {

using tc::fence_after_sync;
using tc::fence_before_sync;
using tc::fence_smem_to_async;
using tc::mbar_arrive;
using tc::mbar_init;
using tc::mbar_wait_bounded;
using tc::mma_bf16_tmem;
using tc::mma_commit;
using tc::sdesc;
using tc::tmem_alloc;
using tc::tmem_dealloc;
using tc::tmem_ld32;

constexpr int TX = 8, TY = 16;                 // tile of one z-plane: 128 cells
constexpr int HX = TX + 2, HY = TY + 2, HZ = 4;  // halo; the 4th plane feeds the discarded row block
constexpr int Z = HX * HY;                     // 180 cells per halo plane
constexpr int HC = Z * HZ;                     // 720 cells per chunk plane
constexpr int CH = 32;
constexpr int NCHUNK = 4;
constexpr int NTHREADS = 288, NLOAD = 256;
constexpr int NBUF = 2;
constexpr uint32_t TMEM_COLS = 512;  // 9 x 32 used
constexpr size_t X_BYTES = (size_t)NCHUNK * HC * 16;         // 46,080
constexpr size_t Y_BYTES = (size_t)NCHUNK * TX * TY * 16;    // 8,192
constexpr size_t BUF_BYTES = X_BYTES + Y_BYTES;
constexpr size_t SMEM_BYTES = NBUF * BUF_BYTES + 128;

// kind::f16, D FP32, A and B BF16, both MN-major (bits 15, 16), N = 32, M = 128
constexpr uint32_t kIdescW = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(CH >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);

// x halo (chunk-major over 4 planes: chunk q of halo cell c at (q HC + c) 16)
// and the dy tile (chunk q of tile cell t at (q 128 + t) 16) of the one-plane
// tile at (x0, y0, z0); this thread's cp.async copies.  Consecutive threads
// take consecutive chunks of a cell, then of the next cell, so a warp reads
// whole cells and every 32-byte sector it touches is used whole.
__device__ __forceinline__ void tile_async(unsigned char* buf, const __nv_bfloat16* __restrict__ x,
                                           const __nv_bfloat16* __restrict__ dy, int x0, int y0, int z0, int D, int H,
                                           int W) {
    for (int idx = threadIdx.x; idx < HC * NCHUNK; idx += NLOAD) {
        const int q = idx % NCHUNK, c = idx / NCHUNK;
        const int hx = c % HX, rr = c / HX, hy = rr % HY, hz = rr / HY;
        int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;  // gz in [-1, z0 + 2]
        gx += gx < 0 ? W : (gx >= W ? -W : 0);
        gy += gy < 0 ? H : (gy >= H ? -H : 0);
        gz += gz < 0 ? D : 0;
        gz -= gz >= D ? D : 0;
        gz -= gz >= D ? D : 0;  // D == 1: z0 + 2 wraps twice
        const size_t g = ((size_t)gx + (size_t)W * ((size_t)gy + (size_t)H * gz)) * CH + 8 * q;
        const uint32_t dst = smem_u32(buf + (size_t)(q * HC + c) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(x + g) : "memory");
    }
    unsigned char* ybuf = buf + X_BYTES;
    for (int idx = threadIdx.x; idx < TX * TY * NCHUNK; idx += NLOAD) {
        const int q = idx % NCHUNK, t = idx / NCHUNK;
        const int tx = t % TX, ty = t / TX;
        const size_t g = ((size_t)(x0 + tx) + (size_t)W * ((size_t)(y0 + ty) + (size_t)H * z0)) * CH + 8 * q;
        const uint32_t dst = smem_u32(ybuf + (size_t)(q * (TX * TY) + t) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(dy + g) : "memory");
    }
}

// Partial weight gradients: ws[block][tap][i][o] (FP32), one block per CTA
// (gridDim.x blocks; a CTA without tiles writes zeros).  H % 16 == 0,
// W % 8 == 0, any D.
__global__ void __launch_bounds__(NTHREADS, 1)
    conv_wgrad_tc_kernel(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ dy,
                         float* __restrict__ ws, int D, int H, int W, unsigned int* timeouts) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* buf[NBUF] = {smem, smem + BUF_BYTES};
    // mbarriers: tile full [0, 1], tile empty [2, 3], all MMAs done [4]
    uint64_t* mb = reinterpret_cast<uint64_t*>(smem + NBUF * BUF_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mb + 5);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto bar = [&](int k) -> uint32_t { return smem_u32(mb + k); };
    if (warp == 8) tmem_alloc(smem_u32(tslot), TMEM_COLS);
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(bar(b), NLOAD);
            mbar_init(bar(2 + b), 1);
        }
        mbar_init(bar(4), 1);
        *abort = 0;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;

    const int ntx = W / TX, nty = H / TY;
    const int ntiles = ntx * nty * D;
    const int G = gridDim.x;
    const int nmine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / G + 1 : 0;
    auto origin = [&](int i, int& x0, int& y0, int& z0) {
        const int tile = blockIdx.x + i * G;
        const int tx = tile % ntx, r = tile / ntx;
        x0 = tx * TX;
        y0 = (r % nty) * TY;
        z0 = r / nty;
    };
    bool ok = true;
    if (warp == 8) {
        if (lane == 0) {
            for (int i = 0; i < nmine; ++i) {
                const int b = i & 1;
                if (!mbar_wait_bounded(bar(b), (uint32_t)((i >> 1) & 1), abort, timeouts)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t xs = smem_u32(buf[b]), ys = xs + (uint32_t)X_BYTES;
                // A: 16 row groups (chunk, z-plane) Z cells apart; K: x-runs one halo row apart
                const uint64_t a_base = sdesc(xs, HX * 16, Z * 16);
                // B: 4 row groups (chunks) 128 cells apart; K: x-runs 8 cells apart
                const uint64_t b_base = sdesc(ys, TX * 16, TX * TY * 16);
#pragma unroll
                for (int r = 0; r < 9; ++r) {
                    const int cr = (r % 3) + HX * (r / 3);  // (dx+1) + HX (dy+1)
#pragma unroll
                    for (int k = 0; k < TY / 2; ++k)
                        mma_bf16_tmem(tbase + (uint32_t)(r * CH), a_base + (uint64_t)(cr + 2 * k * HX),
                                      b_base + (uint64_t)(2 * k * TX), kIdescW, (i > 0 || k > 0) ? 1u : 0u);
                }
                mma_commit(bar(2 + b));  // tile buffer free
            }
            if (ok && nmine > 0) mma_commit(bar(4));  // every MMA of this CTA done
        }
        __syncwarp();
    } else {
        auto load = [&](int i) {
            int a, b, c;
            origin(i, a, b, c);
            tile_async(buf[i & 1], x, dy, a, b, c, D, H, W);
        };
        auto publish = [&](int i) {
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            fence_smem_to_async();
            mbar_arrive(bar(i & 1));
        };
        for (int i = 0; i < nmine; ++i) {
            if (i >= 2 && !mbar_wait_bounded(bar(2 + (i & 1)), (uint32_t)(((i >> 1) - 1) & 1), abort, timeouts)) {
                ok = false;
                break;
            }
            load(i);
            publish(i);
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        // partials: warp w (< 4) holds TMEM lanes 32 w .. = row groups (q = w,
        // z' = lane / 8), channel i = 8 w + lane % 8; dz = z' - 1 (z' = 3 discarded)
        if (warp < 4) {
            float* wsb = ws + (size_t)blockIdx.x * 27 * CH * CH;
            const int zp = lane >> 3, ich = 8 * warp + (lane & 7);
            const bool have = ok && nmine > 0 && mbar_wait_bounded(bar(4), 0u, abort, timeouts);
            if (have) fence_after_sync();
#pragma unroll 1
            for (int r = 0; r < 9; ++r) {
                float v[32];
                if (have) {
                    tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(r * CH), v);
                } else {
#pragma unroll
                    for (int o = 0; o < 32; ++o) v[o] = 0.f;
                }
                if (zp < 3) {
                    float4* p = reinterpret_cast<float4*>(wsb + ((size_t)(zp * 9 + r) * CH + ich) * CH);
#pragma unroll
                    for (int o4 = 0; o4 < 8; ++o4) p[o4] = make_float4(v[4 * o4], v[4 * o4 + 1], v[4 * o4 + 2], v[4 * o4 + 3]);
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 8) tmem_dealloc(tbase, TMEM_COLS);
}

}  // namespace wtc
}  // namespace sur
