// gs_dcpse.cuh -- Gray-Scott with the DC-PSE Laplacian (the operator of the
// paper's Gray-Scott benchmark, which cites the discretization-corrected
// particle strength exchange of Schrader et al.) on the regular grid.
//
// On a regular grid every cell has the same neighbourhood, so the DC-PSE
// Laplacian is one stencil: L f_p = sum_q w_q (f_{p+o_q} - f_p) over the
// integer offsets o_q with |o_q| <= r_c (122 of them at r_c = 3.1 spacings).
// The host solves the moment system for the weights once per context
// (gs_grid.cu); they travel as a kernel parameter (constant bank, broadcast
// to every thread).
//
// dcpse_stage_kernel: one stage k_i = F(Y_i) on a tile of 8 x 8 x TZ
// cells (TZ = 8 or 4): the CTA loads Y_i on the tile plus a halo of R = 3
// cells ((TZ + 6) x 14 x 14 values per component) into shared memory, then
// each thread sums its cell's stencil from there.  Y_i is formed once per
// cell by the stage before (Y_1 = u): at its own cell a stage also forms the
// next stage's input Y_{i+1} = u + dt sum_{j<=i} a_{i+1,j} k_j from u,
// k_1..k_{i-1} and the k_i it has just computed, and the last stage forms
// u' = u + dt sum_j b_j k_j and, for an error-controlled attempt, the
// maximum over cells of |dt sum_j e_j k_j| / (atol + rtol (|u| + dt |k1|)).
// So every field value is formed once, and a step is s launches.
//
// The kernel takes any tableau (up to the 13 stages of Fehlberg 7(8)) and
// any stencil of the form above; it also serves the Cash-Karp and Fehlberg
// steppers with the 7-point Laplacian, written as the stencil of its six
// neighbours (w = 1 / h_d^2) with a halo of R = 1.
#pragma once

#include "gs_tile.cuh"

namespace gsk {

constexpr int kDcpseMax = 256;   // stencil entries (r_c < 4 spacings)
constexpr int kDcpseR = 3;       // halo of the DC-PSE tile (r_c < 4)
constexpr int kDcpseT = 8;       // tile edge
constexpr int kDcpseMaxNK = 12;  // stage inputs (Fehlberg 7(8) stage 13 reads k1..k12)
constexpr int kTabMaxS = kDcpseMaxNK + 1;

// edge of the shared-memory tile of halo R
__host__ __device__ constexpr int tile_edge(int R) { return kDcpseT + 2 * R; }

// The weights are even in the offset (w_{-o} = w_o: the moment system is
// symmetric under o -> -o, and the host averages the two solved values), so
// the FP64 kernel sums the stencil over the npair pairs {o, -o}:
// L f_p = sum_k w_k (f_{p+o_k} + f_{p-o_k}) - wsum f_p, wsum = sum_q w_q:
// one add and one FMA per pair instead of a subtract and an FMA per
// neighbour, half the FP64 operations (the bound of the FP64 kernel).  The
// rounding differs from the per-neighbour form by a few ulp of sum |w| |f|.
// The FP32 kernel keeps the per-neighbour differences (FP32 arithmetic is
// not its bound, and the differences keep its rounding small).
template <typename T>
struct DcpseStencil {
    int count;
    signed char off[kDcpseMax][3];
    T w[kDcpseMax];
    int npair;
    short pidx[kDcpseMax / 2];  // offset of pair k in the flattened Ys tile: (oz E + oy) E + ox, E = tile_edge(R)
    T pw[kDcpseMax / 2];
    T wsum;
};

template <typename T>
struct DcpseStageArgs {
    const T* y[2];               // stage input Y_i (read with the halo)
    const T* u[2];               // state (own cell: next input and final combination)
    const T* k[kDcpseMaxNK][2];  // k_1..k_{i-1} (own cell)
    int nk;                      // i - 1
    double dt;
    T* out[2];                   // k_i
    // next stage input (yn[0] != nullptr): Y_{i+1} = u + dt sum_{j<=i} an_j k_j
    double an[kDcpseMaxNK + 1];
    T* yn[2];
    // last stage (fin != nullptr): fin = u + dt sum_{j<=i} b_j k_j and, with
    // emax, the scaled error maximum (bits of a non-negative double)
    double b[kDcpseMaxNK + 1];
    double e[kDcpseMaxNK + 1];
    double atol, rtol;
    T* fin[2];
    unsigned long long* emax;
};

template <typename T, int TZ, int R>
__global__ void __launch_bounds__(64 * TZ) dcpse_stage_kernel(const Geom<T> g, const DcpseStencil<T> S,
                                                              const DcpseStageArgs<T> A) {
    constexpr int kDcpseE = tile_edge(R);
    constexpr int EZ = TZ + 2 * R;
    __shared__ T Ys[2][EZ][kDcpseE][kDcpseE];
    __shared__ double red[32];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int tilesx = (nx + kDcpseT - 1) / kDcpseT, tilesy = (ny + kDcpseT - 1) / kDcpseT;
    const int bx = blockIdx.x % tilesx, by = (blockIdx.x / tilesx) % tilesy, bz = blockIdx.x / (tilesx * tilesy);
    const int x0 = bx * kDcpseT, y0 = by * kDcpseT, z0 = bz * TZ;
    const int tid = threadIdx.x;
    // Y_i on the tile and its halo (periodic)
    for (int e = tid; e < EZ * kDcpseE * kDcpseE; e += blockDim.x) {
        const int ex = e % kDcpseE, ey = (e / kDcpseE) % kDcpseE, ez = e / (kDcpseE * kDcpseE);
        int x = x0 + ex - R, y = y0 + ey - R, z = z0 + ez - R;
        x = ((x % nx) + nx) % nx;
        y = ((y % ny) + ny) % ny;
        z = ((z % nz) + nz) % nz;
        const long long i = (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
        Ys[0][ez][ey][ex] = A.y[0][i];
        Ys[1][ez][ey][ex] = A.y[1][i];
    }
    __syncthreads();
    const int lx = tid % kDcpseT, ly = (tid / kDcpseT) % kDcpseT, lz = tid / (kDcpseT * kDcpseT);
    const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
    const bool valid = x < nx && y < ny && z < nz;
    double emax = 0.0;
    if (valid) {
        const int cx = lx + R, cy = ly + R, cz = lz + R;
        const T yu = Ys[0][cz][cy][cx], yv = Ys[1][cz][cy][cx];
        T lu = T(0), lv = T(0);
        if constexpr (sizeof(T) == 8) {
            const T* pu = &Ys[0][cz][cy][cx];
            const T* pv = &Ys[1][cz][cy][cx];
#pragma unroll 4
            for (int k = 0; k < S.npair; ++k) {
                const int o = S.pidx[k];
                lu = fma(S.pw[k], pu[o] + pu[-o], lu);
                lv = fma(S.pw[k], pv[o] + pv[-o], lv);
            }
            lu = fma(-S.wsum, yu, lu);
            lv = fma(-S.wsum, yv, lv);
        } else {
            for (int q = 0; q < S.count; ++q) {
                const int ox = S.off[q][0], oy = S.off[q][1], oz = S.off[q][2];
                lu += S.w[q] * (Ys[0][cz + oz][cy + oy][cx + ox] - yu);
                lv += S.w[q] * (Ys[1][cz + oz][cy + oy][cx + ox] - yv);
            }
        }
        const T uvv = yu * yv * yv;
        T f[2];
        f[0] = g.Du * lu - uvv + g.F * (T(1) - yu);
        f[1] = g.Dv * lv + uvv - (g.F + g.k) * yv;
        const long long i = (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
        const T dt = (T)A.dt;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            A.out[c][i] = f[c];
            if (A.yn[0]) {
                // Y_{i+1} = u + dt (sum_j an_j k_j), summed from k_1 up
                T s = T(0);
                for (int j = 0; j < A.nk; ++j) s = (j == 0) ? (T)A.an[0] * A.k[j][c][i] : s + (T)A.an[j] * A.k[j][c][i];
                s = (A.nk == 0) ? (T)A.an[0] * f[c] : s + (T)A.an[A.nk] * f[c];
                A.yn[c][i] = A.u[c][i] + dt * s;
            }
            if (A.fin[0]) {
                // u' = u + dt sum_j b_j k_j and the error terms, in FP64
                const double u = (double)A.u[c][i];
                double sb = 0.0, se = 0.0, k1 = 0.0;
                for (int j = 0; j <= A.nk; ++j) {
                    const double kj = (j < A.nk) ? (double)A.k[j][c][i] : (double)f[c];
                    if (j == 0) k1 = kj;
                    sb += A.b[j] * kj;
                    se += A.e[j] * kj;
                }
                A.fin[c][i] = (T)(u + A.dt * sb);
                if (A.emax) {
                    const double sc = A.atol + A.rtol * (fabs(u) + A.dt * fabs(k1));
                    emax = nanmax(emax, fabs(A.dt * se) / sc);
                }
            }
        }
    }
    if (A.emax) {  // uniform over the launch: every thread reaches the block reduction
        const double bmax = block_nanmax(emax, red);
        if (tid == 0) atomic_max_nonneg(A.emax, bmax);
    }
}

// u' = u + dt sum_j b_j k_j as its own pass (Euler: its one stage reads u
// with the halo, so the update cannot overwrite u inside that stage)
template <typename T>
struct DcpseCombineArgs {
    const T* u[2];
    const T* k[kTabMaxS][2];
    double b[kTabMaxS];
    double e[kTabMaxS];  // error weights (if emax != nullptr)
    int nk;
    double dt, atol, rtol;
    T* out[2];
    unsigned long long* emax;  // bits of the maximum scaled error (NaN sorts high)
};

template <typename T>
__global__ void __launch_bounds__(256) dcpse_combine_kernel(long long n, const DcpseCombineArgs<T> A) {
    __shared__ double red[32];
    double emax = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const double u = (double)A.u[c][i];
            double s = 0.0, e = 0.0;
            for (int j = 0; j < A.nk; ++j) {
                const double kj = (double)A.k[j][c][i];
                s += A.b[j] * kj;
                e += A.e[j] * kj;
            }
            A.out[c][i] = (T)(u + A.dt * s);
            if (A.emax) {
                const double sc = A.atol + A.rtol * (fabs(u) + A.dt * fabs((double)A.k[0][c][i]));
                emax = nanmax(emax, fabs(A.dt * e) / sc);
            }
        }
    }
    if (A.emax) {
        const double bmax = block_nanmax(emax, red);
        if (threadIdx.x == 0) atomic_max_nonneg(A.emax, bmax);
    }
}

}  // namespace gsk
