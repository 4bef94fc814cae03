// gs_tile.cuh -- the fused Gray-Scott stage kernel.
//
// One launch evaluates one Runge-Kutta stage over the whole grid in a single
// pass over HBM:
//   Y   = u + dt * sum_j a_j k_j          (stage input, formed on the fly)
//   f   = F(Y)                            (Gray-Scott right-hand side, Eq. 2:
//                                          7-point periodic Laplacian + u v^2
//                                          reaction, v-equation of Listing 2)
//   epilogue, one of
//     STAGE       : write f                         (k_i of the next stage)
//     FINAL       : write u + dt (sum bk k + sum be ex + bf f) [and f]
//                   (RK4 / Euler / Adams-Bashforth update, history write)
//     DOPRI_FINAL : write Y (= the 5th-order solution) and f (= k7, reused as
//                   the next k1), and reduce the scaled error norm.
//
// Tiling: persistent CTAs own equal shares of the (column, z-plane) space;
// a column is 30 (x) by ty (y) interior cells.  A CTA has 32 x (ty + 2) threads: lane L covers
// column x0 - 1 + L and warp w covers row y0 - 1 + w, so lanes 0 and 31 and
// warps 0 and ty+1 load the xy-halo while the interior threads compute.  Y of
// the current plane and its two z-neighbours live in a 4-slot shared-memory
// ring (one __syncthreads per plane), so each input is read once per plane
// (plus the halo, which adjacent CTAs read from L2).
//
// Final kernels optionally run the step-size controller in the last CTA to
// finish (arrival counter in the control block), and set the CUDA-graph
// conditional that drives the step loop, so a whole integration runs without
// host round trips.
#pragma once

#include "common.cuh"

namespace gsk {

// MODE_DOPRI_S6 / S7: the Dormand-Prince stages 6 and 7 with the work split
// differently (staged form only): stage 6 also forms y5 (b7 = 0, so y5 needs
// k1..k6 only), the error terms of k1..k6 and the inverse error scale, and
// never stores k6; stage 7 evaluates k7 = F(y5) and adds its error term.
// MODE_PAIR_STAGE / MODE_PAIR_DOPRI23 / MODE_PAIR_DOPRI45 /
// MODE_PAIR_DOPRI67 / MODE_PAIR_RK4: two consecutive stages in one launch
// (gs_pair.cuh): stages i and i+1; Dormand-Prince stages 2 and 3 that also
// write the inverse error scale; stages 4 and 5 writing stage 6's input, the
// partial y5 and the error terms through k5 instead of k4 and k5; stages 6
// and 7 from those fields with y5, k7 and the error norm; RK4 stages 3 and 4
// with the update.
enum StageMode : int {
    MODE_STAGE = 0,
    MODE_FINAL = 1,
    MODE_DOPRI_FINAL = 2,
    MODE_DOPRI_S6 = 3,
    MODE_DOPRI_S7 = 4,
    MODE_PAIR_STAGE = 5,
    MODE_PAIR_DOPRI67 = 6,
    MODE_PAIR_RK4 = 7,
    MODE_PAIR_DOPRI45 = 8,
    MODE_PAIR_DOPRI23 = 9
};

template <typename T>
struct Geom {
    int nx, ny, nz;
    T cx, cy, cz;  // 1 / h_d^2
    T Du, Dv, F, k;
};

constexpr int kTileX = 30;      // interior columns per CTA (32 lanes incl. 2 halo)
constexpr int kMaxNK = 5;       // stage inputs combined into Y
constexpr int kMaxNE = 3;       // pointwise inputs of a final combination
constexpr int kMaxTY = 14;      // rows per tile (CTA = 32 x (ty+2) <= 512 threads)
constexpr int kMaxTYFinal = 6;  // final kernels: CTA <= 256 threads (more registers per thread)

struct StageArgs {
    Slot u;                 // state the stage starts from
    Slot kin[kMaxNK];       // stage inputs (read with halo)
    double a[kMaxNK];       // Y = u + dt * sum_j a[j] kin[j]
    Slot ex[kMaxNE];        // pointwise inputs of a FINAL combination
    double bk[kMaxNK];      // FINAL: u + dt (sum bk_j kin_j + sum be_j ex_j + bf f)
    double be[kMaxNE];
    double bf;
    Slot out0, out1;
    Slot out2;              // MODE_DOPRI_S6, MODE_PAIR_DOPRI23: inverse error scale; MODE_PAIR_DOPRI45: error terms
    int n_ex;
    int has_out1;
    int ty, zc;             // tile shape
    int ntx, nty, ntz;      // tile counts
    int kper;               // > 0: column-split schedule with kper z-bands per column
    DevCtrl* ctrl;          // may be null: plain F evaluation with dt = 0
    int run_ctrl;           // final kernels: run the controller in the last CTA
    unsigned long long cond;  // cudaGraphConditionalHandle (valid if use_cond)
    int use_cond;
};

template <typename T>
__host__ __device__ inline size_t stage_smem_bytes(int ty) {
    return sizeof(T) * 4 * (size_t)(ty + 2) * 2 * 32;
}

template <typename T, int NK>
struct CellIn {
    T u[2];
    T k[NK > 0 ? NK : 1][2];
};

__device__ __forceinline__ int wrap1(int a, int n) {
    // a in [-1, n]
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

template <typename T, int NK, int MODE>
__global__ void __launch_bounds__(MODE == MODE_STAGE ? 512 : 256) gs_stage_kernel(const Geom<T> g, const StageArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    __shared__ T red[32];
    __shared__ int s_last;

    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int TY = A.ty;
    const int TYP = TY + 2;

    int parity = 0;
    long long step = 0;
    double dtd = 0.0, atol = 0.0, rtol = 0.0;
    int skip = 0;
    if (A.ctrl) {
        parity = A.ctrl->parity;
        step = A.ctrl->step;
        dtd = A.ctrl->dt_try;
        atol = A.ctrl->atol;
        rtol = A.ctrl->rtol;
        skip = A.ctrl->done;
    }
    const T dt = (T)dtd;

    const T* __restrict__ uin[2] = {resolve<T>(A.u, 0, parity, step), resolve<T>(A.u, 1, parity, step)};
    const T* kin[NK > 0 ? NK : 1][2];
    T aT[NK > 0 ? NK : 1];
#pragma unroll
    for (int j = 0; j < NK; ++j) {
        kin[j][0] = resolve<T>(A.kin[j], 0, parity, step);
        kin[j][1] = resolve<T>(A.kin[j], 1, parity, step);
        aT[j] = (T)A.a[j];
    }
    T* o0[2] = {resolve<T>(A.out0, 0, parity, step), resolve<T>(A.out0, 1, parity, step)};
    const T* exs[kMaxNE][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    if (MODE == MODE_FINAL) {
        for (int j = 0; j < A.n_ex; ++j) {
            exs[j][0] = resolve<T>(A.ex[j], 0, parity, step);
            exs[j][1] = resolve<T>(A.ex[j], 1, parity, step);
        }
    }
    T* o1[2] = {nullptr, nullptr};
    if (MODE != MODE_STAGE && A.has_out1) {
        o1[0] = resolve<T>(A.out1, 0, parity, step);
        o1[1] = resolve<T>(A.out1, 1, parity, step);
    }

    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long plane = (long long)nx * ny;
    T emax = T(0);

    auto sidx = [&](int slot, int ww, int c, int ll) -> int {
        return (((slot & 3) * TYP + ww) * 2 + c) * 32 + ll;
    };
    auto load = [&](long long idx, CellIn<T, NK>& in) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            in.u[c] = __ldg(uin[c] + idx);
#pragma unroll
            for (int j = 0; j < NK; ++j) in.k[j][c] = __ldg(kin[j][c] + idx);
        }
    };
    auto stageY = [&](const CellIn<T, NK>& in, int c) -> T {
        if (NK == 0) return in.u[c];
        T s = aT[0] * in.k[0][c];
#pragma unroll
        for (int j = 1; j < NK; ++j) s += aT[j] * in.k[j][c];
        return in.u[c] + dt * s;
    };

    if (!skip) {
        // schedule (host-chosen): kper > 0 -- column-split: column b % ncols,
        // z-band b / ncols of kper equal bands, so every column advances
        // through the same planes in step and halos are shared through L2;
        // kper == 0 -- CTA b owns planes [L b / G, L (b+1) / G) of the
        // linearised (column, z) space, L = columns * nz, cut at column ends
        const int ncols = A.ntx * A.nty;
        const long long L = A.kper > 0 ? (long long)ncols * A.kper : (long long)ncols * nz;
        const long long s_end = A.kper > 0 ? blockIdx.x + 1 : L * (blockIdx.x + 1) / gridDim.x;
        for (long long sg = A.kper > 0 ? blockIdx.x : L * blockIdx.x / gridDim.x; sg < s_end;) {
            int col, z0, z1;
            if (A.kper > 0) {
                col = (int)(sg % ncols);
                const int band = (int)(sg / ncols);
                z0 = (int)((long long)band * nz / A.kper);
                z1 = (int)((long long)(band + 1) * nz / A.kper);
                sg += 1;
                if (band >= A.kper || z0 >= z1) continue;
            } else {
                col = (int)(sg / nz);
                z0 = (int)(sg - (long long)col * nz);
                z1 = (int)min((long long)nz, z0 + (s_end - sg));
                sg += z1 - z0;
            }
            const int tx = col % A.ntx;
            const int tyi = col / A.ntx;
            const int x0 = tx * kTileX, y0 = tyi * TY;
            const int aw = min(kTileX, nx - x0);
            const int ah = min(TY, ny - y0);
            const bool act = (lane <= aw + 1) && (w <= ah + 1);
            const bool inner = (lane >= 1) && (lane <= aw) && (w >= 1) && (w <= ah);
            const int x = wrap1(x0 - 1 + lane, nx);
            const int y = wrap1(y0 - 1 + w, ny);
            const long long colrow = (long long)x + (long long)nx * y;

            CellIn<T, NK> cur, nxt;
            if (act) {
                CellIn<T, NK> pre;
                load(colrow + plane * wrap1(z0 - 1, nz), pre);
                S[sidx(0, w, 0, lane)] = stageY(pre, 0);
                S[sidx(0, w, 1, lane)] = stageY(pre, 1);
                load(colrow + plane * z0, cur);
                S[sidx(1, w, 0, lane)] = stageY(cur, 0);
                S[sidx(1, w, 1, lane)] = stageY(cur, 1);
            }
            for (int z = z0; z < z1; ++z) {
                const int r = z - z0 + 1;
                if (act) {
                    load(colrow + plane * wrap1(z + 1, nz), nxt);
                    S[sidx(r + 1, w, 0, lane)] = stageY(nxt, 0);
                    S[sidx(r + 1, w, 1, lane)] = stageY(nxt, 1);
                }
                __syncthreads();
                if (inner) {
                    T Yc[2], lap[2];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const T yc = S[sidx(r, w, c, lane)];
                        const T xm = S[sidx(r, w, c, lane - 1)];
                        const T xp = S[sidx(r, w, c, lane + 1)];
                        const T ym = S[sidx(r, w - 1, c, lane)];
                        const T yp = S[sidx(r, w + 1, c, lane)];
                        const T zm = S[sidx(r - 1, w, c, lane)];
                        const T zp = S[sidx(r + 1, w, c, lane)];
                        Yc[c] = yc;
                        lap[c] = (xm - T(2) * yc + xp) * g.cx + (ym - T(2) * yc + yp) * g.cy +
                                 (zm - T(2) * yc + zp) * g.cz;
                    }
                    const T uvv = Yc[0] * Yc[1] * Yc[1];
                    T f[2];
                    f[0] = g.Du * lap[0] - uvv + g.F * (T(1) - Yc[0]);
                    f[1] = g.Dv * lap[1] + uvv - (g.F + g.k) * Yc[1];
                    const long long i = colrow + plane * z;

                    if (MODE == MODE_STAGE) {
                        o0[0][i] = f[0];
                        o0[1][i] = f[1];
                    } else if (MODE == MODE_FINAL) {
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            T s = (T)A.bf * f[c];
#pragma unroll
                            for (int j = 0; j < NK; ++j) s += (T)A.bk[j] * cur.k[j][c];
#pragma unroll
                            for (int j = 0; j < kMaxNE; ++j)
                                if (j < A.n_ex) s += (T)A.be[j] * exs[j][c][i];
                            o0[c][i] = cur.u[c] + dt * s;
                            if (A.has_out1) o1[c][i] = f[c];
                        }
                    } else {  // MODE_DOPRI_FINAL: kin = {k1, k3, k4, k5, k6}
                        const T ta = (T)atol, tr = (T)rtol;
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            o0[c][i] = Yc[c];
                            o1[c][i] = f[c];
                            if (NK == 5) {
                                const T k1 = cur.k[0][c];
                                // sum_j e_j k_j = sum_j e_j (k_j - k1) since sum_j e_j = 0;
                                // the differences are exact in floating point when close.
                                const T es = (T)dp5::E3 * (cur.k[1][c] - k1) +
                                             (T)dp5::E4 * (cur.k[2][c] - k1) +
                                             (T)dp5::E5 * (cur.k[3][c] - k1) +
                                             (T)dp5::E6 * (cur.k[4][c] - k1) +
                                             (T)dp5::E7 * (f[c] - k1);
                                const T err = dt * es;
                                const T sc = ta + tr * (fabs(cur.u[c]) + dt * fabs(k1));
                                emax = nanmax(emax, (T)(fabs(err) / sc));
                            }
                        }
                    }
                }
                cur = nxt;
            }
            __syncthreads();  // smem ring reused by the next tile
        }
    }

    if (MODE != MODE_STAGE && A.run_ctrl && A.ctrl) {
        const int tid = threadIdx.x + blockDim.x * threadIdx.y;
        if (MODE == MODE_DOPRI_FINAL) {
            const T bmax = block_nanmax(emax, red);
            if (tid == 0) atomic_max_nonneg(&A.ctrl->err_bits, (double)bmax);
        }
        if (tid == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(&A.ctrl->arrive, 1u);
            s_last = (prev == gridDim.x - 1) ? 1 : 0;
        }
        __syncthreads();
        if (s_last && tid == 0) {
            __threadfence();
            DevCtrl* c = A.ctrl;
            const double E = __longlong_as_double((long long)atomicOr(&c->err_bits, 0ull));
            c->err_bits = 0ull;
            c->arrive = 0u;
            int cont = 0;
            if (!c->done) cont = controller_update(c, E);
            if (A.use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)A.cond, cont ? 1u : 0u);
        }
    }
}

}  // namespace gsk
