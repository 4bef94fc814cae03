// gs_persist.cuh -- fixed-step RK4 for small grids in ONE cooperative launch.
//
// A small grid (a few hundred thousand cells) keeps all its fields in L2,
// and a step of four stage kernels is then bound by launch and drain
// latency rather than by memory.  This kernel runs all steps of a call in
// one cooperative launch (every CTA resident): each CTA takes cells in a
// grid-stride loop, and a grid barrier separates the stages (a stage reads
// the previous stage's output at the six neighbours).  The formulas and
// their summation order are those of the stage kernels: Y = u + dt (a k),
// k_s = F(Y) (7-point periodic Laplacian + reaction), u' = u + dt (k4/6 +
// k3/3 + k1/6 + k2/3).  The state ping-pongs between the caller's arrays and
// the context's second buffer; after an odd number of steps it is copied
// back.
//
// Values written by other CTAs in the previous stage are read with L2-only
// loads (__ldcg), so no SM can see a stale line of its own L1.
//
// The grid barrier is a generation counter in global memory: the last CTA
// to arrive resets the count and advances the generation; the others poll
// it.  Every poll loop has an iteration limit: on expiry the CTA sets the
// error word and every CTA leaves at its next barrier (the host reports
// GS_ERR_CUDA).
#pragma once

#include "gs_tile.cuh"

namespace gsk {

constexpr long kBarrierPolls = 1L << 24;

template <typename T>
struct RK4Bufs {
    T* s[2][2];  // [buffer][component]: 0 = caller's state, 1 = the context's second buffer
    T* k[3][2];  // k1, k2, k3
};

// bar[0]: arrival count, bar[1]: generation, bar[2]: error (nonzero: stop)
__device__ __forceinline__ bool grid_sync_bounded(unsigned* bar) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        volatile unsigned* verr = bar + 2;
        const unsigned g = *vgen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long it = 0;
            while (*vgen == g) {
                if (*verr) {
                    ok = 0;
                    break;
                }
                if (++it > kBarrierPolls) {
                    atomicExch(bar + 2, 1u);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok && *verr == 0u;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(256) rk4_persistent_kernel(const Geom<T> g, const RK4Bufs<T> B, const double dtd,
                                                             const long long nsteps, unsigned* bar) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long N = (long long)nx * ny * nz, plane = (long long)nx * ny;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, di = (long long)gridDim.x * blockDim.x;
    const T dt = (T)dtd, half = (T)0.5, one = (T)1;
    const T bf = (T)(1.0 / 6.0), bk0 = (T)(1.0 / 3.0), be0 = (T)(1.0 / 6.0), be1 = (T)(1.0 / 3.0);
    // current and next state (swapped after every step); k1, k2, k3
    T *u0 = B.s[0][0], *u1 = B.s[0][1], *o0 = B.s[1][0], *o1 = B.s[1][1];
    T *a0 = B.k[0][0], *a1 = B.k[0][1], *b0 = B.k[1][0], *b1 = B.k[1][1], *c0 = B.k[2][0], *c1 = B.k[2][1];
    // F at cell i of the stage input Y(j, c) (Y given at any cell j)
    auto rhs = [&](long long i, auto Y, T (&f)[2]) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        const long long xm = x == 0 ? i + nx - 1 : i - 1, xp = x == nx - 1 ? i - nx + 1 : i + 1;
        const long long ym = y == 0 ? i + plane - nx : i - nx, yp = y == ny - 1 ? i - plane + nx : i + nx;
        const long long zm = z == 0 ? i + N - plane : i - plane, zp = z == nz - 1 ? i - N + plane : i + plane;
        T yc[2], lap[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const T yy = Y(i, c);
            yc[c] = yy;
            lap[c] = (Y(xm, c) - T(2) * yy + Y(xp, c)) * g.cx + (Y(ym, c) - T(2) * yy + Y(yp, c)) * g.cy +
                     (Y(zm, c) - T(2) * yy + Y(zp, c)) * g.cz;
        }
        const T uvv = yc[0] * yc[1] * yc[1];
        f[0] = g.Du * lap[0] - uvv + g.F * (T(1) - yc[0]);
        f[1] = g.Dv * lap[1] + uvv - (g.F + g.k) * yc[1];
    };
    for (long long n = 0; n < nsteps; ++n) {
        // k1 = F(u)
        for (long long i = i0; i < N; i += di) {
            T f[2];
            rhs(i, [&](long long j, int c) { return c ? __ldcg(u1 + j) : __ldcg(u0 + j); }, f);
            a0[i] = f[0];
            a1[i] = f[1];
        }
        if (!grid_sync_bounded(bar)) return;
        // k2 = F(u + dt (k1 / 2))
        for (long long i = i0; i < N; i += di) {
            T f[2];
            rhs(i, [&](long long j, int c) {
                return c ? __ldcg(u1 + j) + dt * (half * __ldcg(a1 + j)) : __ldcg(u0 + j) + dt * (half * __ldcg(a0 + j));
            }, f);
            b0[i] = f[0];
            b1[i] = f[1];
        }
        if (!grid_sync_bounded(bar)) return;
        // k3 = F(u + dt (k2 / 2))
        for (long long i = i0; i < N; i += di) {
            T f[2];
            rhs(i, [&](long long j, int c) {
                return c ? __ldcg(u1 + j) + dt * (half * __ldcg(b1 + j)) : __ldcg(u0 + j) + dt * (half * __ldcg(b0 + j));
            }, f);
            c0[i] = f[0];
            c1[i] = f[1];
        }
        if (!grid_sync_bounded(bar)) return;
        // k4 = F(u + dt k3); u' = u + dt (k4/6 + k3/3 + k1/6 + k2/3)
        for (long long i = i0; i < N; i += di) {
            T f[2];
            rhs(i, [&](long long j, int c) {
                return c ? __ldcg(u1 + j) + dt * (one * __ldcg(c1 + j)) : __ldcg(u0 + j) + dt * (one * __ldcg(c0 + j));
            }, f);
            T s0 = bf * f[0], s1 = bf * f[1];
            s0 += bk0 * __ldcg(c0 + i);
            s1 += bk0 * __ldcg(c1 + i);
            s0 += be0 * __ldcg(a0 + i);
            s1 += be0 * __ldcg(a1 + i);
            s0 += be1 * __ldcg(b0 + i);
            s1 += be1 * __ldcg(b1 + i);
            o0[i] = __ldcg(u0 + i) + dt * s0;
            o1[i] = __ldcg(u1 + i) + dt * s1;
        }
        if (!grid_sync_bounded(bar)) return;
        T* t0 = u0;
        T* t1 = u1;
        u0 = o0;
        u1 = o1;
        o0 = t0;
        o1 = t1;
    }
    if (nsteps & 1) {
        for (long long i = i0; i < N; i += di) {
            B.s[0][0][i] = __ldcg(B.s[1][0] + i);
            B.s[0][1][i] = __ldcg(B.s[1][1] + i);
        }
    }
}

}  // namespace gsk
