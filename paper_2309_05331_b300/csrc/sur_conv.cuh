// sur_conv.cuh -- BF16 tensor-core kernels of the learned surrogate: 3x3x3
// periodic convolutions as implicit GEMMs (forward / input gradient) and the
// weight gradient, on channels-last activations with C in {8, 32} channels
// (a 16-byte multiple per cell; 2-channel tensors are stored padded to 8).
//
// Products are BF16 x BF16 with FP32 accumulation (mma.sync m16n8k16).
// Tiles: 16 (x) x 8 (y) x 2 (z) output cells per CTA of 8 warps; each warp
// owns the 16-cell x-rows (y = warp, z = 0 and 1), i.e. two M=16 tiles.  The
// periodic input halo tile (18 x 10 x 4 cells) and the packed weights sit in
// shared memory; 16-byte chunks are XOR-swizzled so every ldmatrix reads 8
// rows from 8 different bank groups.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sur {

constexpr int TX = 16, TY = 8, TZ = 2;
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int HC = HX * HY * HZ;  // 720 halo cells
constexpr int NTHREADS = 256;
constexpr int TILE_CELLS = TX * TY * TZ;  // 256

// epilogues
enum Epi : int { EPI_BIAS_RELU_BF16 = 0, EPI_BIAS_F32 = 1, EPI_MASK_BF16 = 2, EPI_RAW_F32 = 3 };

// number of K steps (16 each) of a layer with C input channels:
// C = 32: two per tap (54); C = 8: one per pair of taps (14, tap 27 = 0)
__host__ __device__ constexpr int ksteps(int C) { return C == 32 ? 54 : 14; }

// byte offset of 16-byte chunk q of cell c in a tile of C-channel cells
template <int C>
__device__ __forceinline__ int cell_off(int c, int q) {
    if (C == 32) return c * 64 + ((q ^ ((c >> 1) & 3)) << 4);
    return c * 16;
}
// byte offset of chunk q (0/1) of packed weight row (ks, n), N = padded Cout
__host__ __device__ __forceinline__ int wrow_off(int ks, int n, int q, int N) {
    return ((ks * N + n) * 2 + (q ^ ((n >> 2) & 1))) << 4;
}

__device__ __forceinline__ int wrapn(int a, int n) { return ((a % n) + n) % n; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm_x4(uint32_t a, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t a, uint32_t& r0, uint32_t& r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t a, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t a, uint32_t& r0, uint32_t& r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}
// D += A (16x16, row) * B (16x8, col), BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Loads the periodic halo tile of C-channel cells around output tile
// (x0, y0, z0) into shared memory (swizzled chunks).
template <int C>
__device__ __forceinline__ void load_halo(unsigned char* Xs, const __nv_bfloat16* __restrict__ src, int x0, int y0,
                                          int z0, int D, int H, int W) {
    constexpr int CH = C / 8;
    for (int idx = threadIdx.x; idx < HC * CH; idx += NTHREADS) {
        const int cell = idx / CH, q = idx - cell * CH;
        const int hx = cell % HX, r = cell / HX, hy = r % HY, hz = r / HY;
        const int gx = wrapn(x0 + hx - 1, W), gy = wrapn(y0 + hy - 1, H), gz = wrapn(z0 + hz - 1, D);
        const size_t g = ((size_t)gx + (size_t)W * ((size_t)gy + (size_t)H * gz)) * C + 8 * q;
        *reinterpret_cast<uint4*>(Xs + cell_off<C>(cell, q)) = __ldg(reinterpret_cast<const uint4*>(src + g));
    }
}

// Implicit-GEMM 3x3x3 periodic convolution.
//   out[p][o] = epi( sum_{tap, i} Wfwd[tap][i][o] x[p + off(tap)][i] )
// CIN, COUT in {8, 32} (padded counts).  wp: packed weights (ksteps(CIN)
// rows of COUT x 16 BF16, swizzled) -- see sur_pack_weights.
// Epilogues: BIAS_RELU_BF16 (hidden layers), BIAS_F32 (last layer, the first
// `out_ch` channels are stored), MASK_BF16 (input gradient times the ReLU
// derivative of mask > 0), RAW_F32 (tests; bias optional).
// Grid: persistent CTAs over tiles; D % 2 == 0, H % 8 == 0, W % 16 == 0.
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(NTHREADS, 2)
    conv_fwd_kernel(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ wp,
                    const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask, void* out, int out_ch,
                    int D, int H, int W) {
    constexpr int KS = ksteps(CIN);
    constexpr int NT = COUT / 8;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* Ws = smem;                                  // KS * COUT * 32 bytes
    unsigned char* Xs = smem + KS * COUT * 32;                 // HC * CIN * 2 bytes
    unsigned char* Zs = Xs + HC * CIN * 2;                     // 16 zero bytes (padded taps)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // weights once per CTA
    for (int i = tid; i < KS * COUT * 2; i += NTHREADS)
        reinterpret_cast<uint4*>(Ws)[i] = __ldg(reinterpret_cast<const uint4*>(wp) + i);
    if (tid == 0) *reinterpret_cast<uint4*>(Zs) = make_uint4(0, 0, 0, 0);
    const int ntx = W / TX, nty = H / TY, ntz = D / TZ;
    const int ntiles = ntx * nty * ntz;
    const int g = lane >> 2, t = lane & 3;
    const int j = lane >> 3;  // ldmatrix matrix index this lane addresses
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tx = tile % ntx, r = tile / ntx, ty = r % nty, tz = r / nty;
        const int x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
        __syncthreads();  // previous tile's reads of Xs are done
        load_halo<CIN>(Xs, x, x0, y0, z0, D, H, W);
        __syncthreads();
        float acc[2][NT][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < NT; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
        const int row = (lane & 7) + 8 * (j & 1);  // A row (cell along x) of this lane
        for (int ks = 0; ks < KS; ++ks) {
            int tap, q;
            if (CIN == 32) {
                tap = ks >> 1;
                q = 2 * (ks & 1) + (j >> 1);
            } else {
                tap = 2 * ks + (j >> 1);
                q = 0;
            }
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int cell = (row + dx + 1) + HX * ((warp + dy + 1) + HY * (mt + dz + 1));
                const uint32_t addr = (tap < 27) ? smem_u32(Xs + cell_off<CIN>(cell, q)) : smem_u32(Zs);
                ldsm_x4(addr, a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
            }
#pragma unroll
            for (int np = 0; np < (NT + 1) / 2; ++np) {
                uint32_t b[4];
                if (NT >= 2) {
                    const int n = 16 * np + 8 * (j >> 1) + (lane & 7);
                    ldsm_x4(smem_u32(Ws + wrow_off(ks, n, j & 1, COUT)), b[0], b[1], b[2], b[3]);
                } else {
                    const int n = lane & 7;
                    ldsm_x2(smem_u32(Ws + wrow_off(ks, n, j & 1, COUT)), b[0], b[1]);
                    b[2] = b[3] = 0u;
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_bf16(acc[mt][2 * np], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[0], b[1]);
                    if (2 * np + 1 < NT)
                        mma_bf16(acc[mt][2 * np + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[2], b[3]);
                }
            }
        }
        // epilogue: rows g, g+8 (x), columns 2t, 2t+1 of each n-tile
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int xg = x0 + g + 8 * hh, yg = y0 + warp, zg = z0 + mt;
                const size_t cell = (size_t)xg + (size_t)W * ((size_t)yg + (size_t)H * zg);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const int o = 8 * nt + 2 * t;
                    float v0 = acc[mt][nt][2 * hh], v1 = acc[mt][nt][2 * hh + 1];
                    if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_BIAS_F32 || (EPI == EPI_RAW_F32 && bias)) {
                        v0 += bias[o];
                        v1 += bias[o + 1];
                    }
                    if (EPI == EPI_BIAS_RELU_BF16) {
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    if (EPI == EPI_MASK_BF16) {
                        const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(mask + cell * COUT + o);
                        if (!(__bfloat162float(m.x) > 0.f)) v0 = 0.f;
                        if (!(__bfloat162float(m.y) > 0.f)) v1 = 0.f;
                    }
                    if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_BF16) {
                        *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(out) + cell * COUT + o) =
                            __floats2bfloat162_rn(v0, v1);
                    } else if (EPI == EPI_BIAS_F32) {
                        float* po = static_cast<float*>(out) + cell * out_ch;
                        if (o < out_ch) po[o] = v0;
                        if (o + 1 < out_ch) po[o + 1] = v1;
                    } else {
                        *reinterpret_cast<float2*>(static_cast<float*>(out) + cell * COUT + o) = make_float2(v0, v1);
                    }
                }
            }
        }
    }
}

// Weight gradient partials: ws[block][tap][i][o] = sum over this CTA's tiles
// of x[p + off(tap)][i] * dy[p][o].  CIN, COUT in {8, 32}.  Warp w owns taps
// w, w+8, w+16, w+24 (< 27).
template <int CIN, int COUT>
__global__ void __launch_bounds__(NTHREADS, 1)
    conv_wgrad_kernel(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ dy,
                      float* __restrict__ ws, int D, int H, int W) {
    constexpr int MT = CIN == 32 ? 2 : 1;
    constexpr int NT = COUT / 8;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* Xs = smem;                     // HC * CIN * 2
    unsigned char* Ys = smem + HC * CIN * 2;      // TILE_CELLS * COUT * 2
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3, j = lane >> 3;
    float acc[4][MT][NT][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < MT; ++b)
#pragma unroll
            for (int c = 0; c < NT; ++c)
#pragma unroll
                for (int d = 0; d < 4; ++d) acc[a][b][c][d] = 0.f;
    const int ntx = W / TX, nty = H / TY, ntz = D / TZ;
    const int ntiles = ntx * nty * ntz;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tx = tile % ntx, r = tile / ntx, ty = r % nty, tz = r / nty;
        const int x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
        __syncthreads();
        load_halo<CIN>(Xs, x, x0, y0, z0, D, H, W);
        constexpr int CHY = COUT / 8;
        for (int idx = tid; idx < TILE_CELLS * CHY; idx += NTHREADS) {
            const int cell = idx / CHY, q = idx - cell * CHY;
            const int cx = cell % TX, rr = cell / TX, cy = rr % TY, cz = rr / TY;
            const size_t gidx = ((size_t)(x0 + cx) + (size_t)W * ((size_t)(y0 + cy) + (size_t)H * (z0 + cz))) * COUT + 8 * q;
            *reinterpret_cast<uint4*>(Ys + cell_off<COUT>(cell, q)) = __ldg(reinterpret_cast<const uint4*>(dy + gidx));
        }
        __syncthreads();
        for (int kk = 0; kk < TY * TZ; ++kk) {  // K step: the 16 cells of one x-row
            const int yy = kk % TY, zz = kk / TY;
            uint32_t b[NT][2];
            {
                // B = dy[cell][o]: rows = cells (k), ldmatrix.trans gives (k pair, n = g)
                const int kcell = (lane & 7) + 8 * (j & 1) + TX * (yy + TY * zz);
#pragma unroll
                for (int np = 0; np < (NT + 1) / 2; ++np) {
                    if (NT >= 2) {
                        ldsm_x4_t(smem_u32(Ys + cell_off<COUT>(kcell, 2 * np + (j >> 1))), b[2 * np][0], b[2 * np][1],
                                  b[2 * np + 1][0], b[2 * np + 1][1]);
                    } else {
                        ldsm_x2_t(smem_u32(Ys + cell_off<COUT>(kcell, 0)), b[0][0], b[0][1]);
                    }
                }
            }
#pragma unroll
            for (int ti = 0; ti < 4; ++ti) {
                const int tap = warp + 8 * ti;
                if (tap >= 27) break;
                const int dz = tap / 9 - 1, dy1 = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                // A = x^T: rows = cells (k) of the shifted x-row, chunk = channel block
                const int kc = (lane & 7) + 8 * (j >> 1);  // cell along x for this lane's matrix
                const int hcell = (kc + dx + 1) + HX * ((yy + dy1 + 1) + HY * (zz + dz + 1));
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    uint32_t a0, a1, a2, a3;
                    if (CIN == 32) {
                        ldsm_x4_t(smem_u32(Xs + cell_off<CIN>(hcell, 2 * mt + (j & 1))), a0, a1, a2, a3);
                    } else {
                        // matrices: lanes 0-7 cells 0-7, lanes 8-15 cells 8-15 (channels 0-7)
                        const int kc2 = (lane & 7) + 8 * (j & 1);
                        const int hc2 = (kc2 + dx + 1) + HX * ((yy + dy1 + 1) + HY * (zz + dz + 1));
                        ldsm_x2_t(smem_u32(Xs + cell_off<CIN>(hc2, 0)), a0, a2);
                        a1 = a3 = 0u;
                    }
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[ti][mt][nt], a0, a1, a2, a3, b[nt][0], b[nt][1]);
                }
            }
        }
    }
    // partials: D rows = input channel i (g, g+8 of m-tile), cols = o (2t, 2t+1)
    float* wsb = ws + (size_t)blockIdx.x * 27 * CIN * COUT;
#pragma unroll
    for (int ti = 0; ti < 4; ++ti) {
        const int tap = warp + 8 * ti;
        if (tap >= 27) break;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int i = 16 * mt + g + 8 * hh;
                    if (i >= CIN) continue;
                    const int o = 8 * nt + 2 * t;
                    float* p = wsb + ((size_t)tap * CIN + i) * COUT + o;
                    p[0] = acc[ti][mt][nt][2 * hh];
                    p[1] = acc[ti][mt][nt][2 * hh + 1];
                }
    }
}

}  // namespace sur
