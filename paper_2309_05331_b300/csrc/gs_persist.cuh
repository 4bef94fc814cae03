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
// The grid barrier: a 64-bit arrival count that is never reset and a
// generation word.  A CTA arrives with an acquire-release add on the count
// (its ticket); the CTA whose ticket completes round r (ticket = (r+1) G - 1)
// publishes generation r+1 with a release add, and the others poll the
// generation with acquire loads.  So a barrier costs one RMW round trip and
// the polls, without full fences or a reset.  Every poll loop has an
// iteration limit: on expiry the CTA sets the error word and every CTA
// leaves at its next barrier (the host reports GS_ERR_CUDA).
#pragma once

#include "gs_tile.cuh"

namespace gsk {

constexpr long kBarrierPolls = 1L << 24;

template <typename T>
struct RK4Bufs {
    T* s[2][2];  // [buffer][component]: 0 = caller's state, 1 = the context's second buffer
    T* k[3][2];  // k1, k2, k3
};

__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;\n" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ void red_add_release_gpu(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// bar: u64 arrival count (bytes 0-7), u32 generation (8-11), u32 error
// (12-15; nonzero: stop).  round: barriers this CTA has passed.
__device__ __forceinline__ bool grid_sync_bounded(unsigned* bar, unsigned& round) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* gen = bar + 2;
        volatile unsigned* verr = bar + 3;
        const unsigned long long nb = gridDim.x;
        const unsigned long long ticket = atom_add_acq_rel_gpu(reinterpret_cast<unsigned long long*>(bar), 1ull);
        const unsigned target = round + 1u;
        int ok = 1;
        if (ticket == (unsigned long long)target * nb - 1ull) {
            red_add_release_gpu(gen, 1u);
        } else {
            long it = 0;
            while ((int)(ld_acquire_gpu(gen) - target) < 0) {
                if (*verr) {
                    ok = 0;
                    break;
                }
                if (++it > kBarrierPolls) {
                    atomicExch(bar + 3, 1u);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok && *verr == 0u;
    }
    __syncthreads();
    ++round;
    return s_ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(256) rk4_persistent_kernel(const Geom<T> g, const RK4Bufs<T> B, const double dtd,
                                                             const long long nsteps, unsigned* bar) {
    // cell indices fit 32 bits (the host takes this path for N < 2^31 only)
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int N = nx * ny * nz, plane = nx * ny;
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x, di = gridDim.x * blockDim.x;
    const T dt = (T)dtd, half = (T)0.5, one = (T)1;
    const T bf = (T)(1.0 / 6.0), bk0 = (T)(1.0 / 3.0), be0 = (T)(1.0 / 6.0), be1 = (T)(1.0 / 3.0);
    // current and next state (swapped after every step); k1, k2, k3
    T *u0 = B.s[0][0], *u1 = B.s[0][1], *o0 = B.s[1][0], *o1 = B.s[1][1];
    T *a0 = B.k[0][0], *a1 = B.k[0][1], *b0 = B.k[1][0], *b1 = B.k[1][1], *c0 = B.k[2][0], *c1 = B.k[2][1];
    unsigned round = 0;  // grid barriers passed
    // F at cell i of the stage input Y(j, c) (Y given at any cell j)
    auto rhs = [&](int i, auto Y, T (&f)[2]) {
        const int r = i / nx, x = i - r * nx;
        const int z = r / ny, y = r - z * ny;
        const int xm = x == 0 ? i + nx - 1 : i - 1, xp = x == nx - 1 ? i - nx + 1 : i + 1;
        const int ym = y == 0 ? i + plane - nx : i - nx, yp = y == ny - 1 ? i - plane + nx : i + nx;
        const int zm = z == 0 ? i + N - plane : i - plane, zp = z == nz - 1 ? i - N + plane : i + plane;
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
        for (int i = i0; i < N; i += di) {
            T f[2];
            rhs(i, [&](int j, int c) { return c ? __ldcg(u1 + j) : __ldcg(u0 + j); }, f);
            a0[i] = f[0];
            a1[i] = f[1];
        }
        if (!grid_sync_bounded(bar, round)) return;
        // k2 = F(u + dt (k1 / 2))
        for (int i = i0; i < N; i += di) {
            T f[2];
            rhs(i, [&](int j, int c) {
                return c ? __ldcg(u1 + j) + dt * (half * __ldcg(a1 + j)) : __ldcg(u0 + j) + dt * (half * __ldcg(a0 + j));
            }, f);
            b0[i] = f[0];
            b1[i] = f[1];
        }
        if (!grid_sync_bounded(bar, round)) return;
        // k3 = F(u + dt (k2 / 2))
        for (int i = i0; i < N; i += di) {
            T f[2];
            rhs(i, [&](int j, int c) {
                return c ? __ldcg(u1 + j) + dt * (half * __ldcg(b1 + j)) : __ldcg(u0 + j) + dt * (half * __ldcg(b0 + j));
            }, f);
            c0[i] = f[0];
            c1[i] = f[1];
        }
        if (!grid_sync_bounded(bar, round)) return;
        // k4 = F(u + dt k3); u' = u + dt (k4/6 + k3/3 + k1/6 + k2/3)
        for (int i = i0; i < N; i += di) {
            T f[2];
            rhs(i, [&](int j, int c) {
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
        if (!grid_sync_bounded(bar, round)) return;
        T* t0 = u0;
        T* t1 = u1;
        u0 = o0;
        u1 = o1;
        o0 = t0;
        o1 = t1;
    }
    if (nsteps & 1) {
        for (int i = i0; i < N; i += di) {
            B.s[0][0][i] = __ldcg(B.s[1][0] + i);
            B.s[0][1][i] = __ldcg(B.s[1][1] + i);
        }
    }
}

}  // namespace gsk
