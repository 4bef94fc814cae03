// gs_pair.cuh -- two consecutive Runge-Kutta stages of the Gray-Scott system
// in one pass over HBM.
//
// Stage i forms Y_i = u + dt sum_{j<i} a_ij k_j and k_i = F(Y_i) (Eq. 2: the
// 7-point periodic Laplacian plus the u v^2 reaction).  Stage i+1 needs
// Y_{i+1} = u + dt sum_{j<=i} a_{i+1,j} k_j at the six neighbours of every
// cell, so k_i is needed on the tile plus a one-cell ring and Y_i on the tile
// plus a two-cell ring.  This kernel computes k_i on that ring (the ring
// cells are also computed by the neighbouring tiles) instead of storing k_i
// and reading it back with a halo in a second launch: the pair reads u and
// k_1..k_{i-1} once and writes k_i and k_{i+1}, i + 3 field passes instead
// of 2i + 3.  Dormand-Prince stages 6 and 7 fuse the same way: stage 7's
// input is y5 = u + dt sum_j b_j k_j (b7 = 0).  Nothing after stage 7 needs
// k4 or k5 themselves, only their pointwise combinations, so the 4+5 pair
// writes, instead of k4 and k5, the three fields stage 6 onwards uses at a
// cell: Y6 = u + dt sum_{j<=5} a_6j k_j, P = u + dt sum_{j<=5} b_j k_j (y5
// without its k6 term) and the error terms through k5; the 2+3 pair, which
// reads u and k1, also writes the inverse error scale 1 / (atol + rtol (|u|
// + dt |k1|)).  The 6+7 pair reads those four fields (Y6 on every row of the
// tile's two-cell ring, P on the one-cell ring, the other two on the tile),
// writes y5 and k7 (the next k1) and reduces the scaled error norm.  An
// attempt still moves 18 field passes (stages 2+3: 5, 4+5: 7, 6+7: 6), but
// the six-array formation of Y6 and P, which the halo rows of the 6+7 tiles
// would repeat, runs once per cell in the 4+5 pair's tile rows.  RK4
// runs as two pairs: k1, k2 from u (stage 1 is F(u)),
// then k3, k4 and the update u' = u + dt (k1/6 + k2/3 + k3/3 + k4/6) from u,
// k1, k2 without storing k3 or k4: 7 field passes per step instead of 13.
//
// Mapping (the staged form's, widened): a warp owns a row of 32*VX cells, a
// vector of VX consecutive cells per lane (16 bytes on the single grid, VX =
// 16 / sizeof(T); the batched ensemble also runs one cell or 8 bytes per
// lane, as its instances' rows allow).  The CTA has ty + 4 row warps for rows
// y0-2 .. y0+ty+1 and one halo warp whose lane 2(r+2)+s owns the two x-halo
// columns of row y0+r on side s (s = 0: x0-2, x0-1; s = 1: x0+aw,
// x0+aw+1).  Planes advance in z with three phases per iteration:
//   A(z+2): Y_i of plane z+2 on every row and halo column, from the inputs;
//           stored in the Y_i plane buffer;
//   B(z+1): k_i of plane z+1 on rows -1..ty and the two inner halo columns
//           (7-point stencil on the Y_i planes z, z+1, z+2), stored for the
//           tile rows (Dormand-Prince 4+5: kept for C; 6+7: y5 stored
//           instead); Y_{i+1} of plane z+1 formed and stored in the Y_{i+1}
//           plane buffer;
//   C(z):   k_{i+1} of plane z on the tile rows, stored (4+5: stage 6's
//           fields instead; 6+7: k7 and the scaled error).
// B reads the Y_i plane that A wrote one iteration earlier (neighbours) and
// its own cells of the plane before (lower z neighbour); C likewise on the
// Y_{i+1} planes.  Three buffers of each and one barrier per iteration order
// every shared-memory access: a buffer is rewritten three iterations after
// it was filled, after the last iteration that reads another thread's cells
// from it.  The upper z neighbour and the centre stay in registers.  The
// inputs arrive through the staged form's per-thread cp.async ring, DEPTH
// planes ahead: every thread copies its own 16-byte vectors (the halo warp
// its 8-byte pairs) with cp.async, and a slot is written and read only by the
// thread that copies it, so cp.async.wait_group is the only ordering the ring
// needs.
#pragma once

#include <type_traits>

#include "gs_staged.cuh"

namespace gsk {

// Tile heights: up to 7 rows in a CTA of 12 warps (3 per SM sub-partition,
// 168 registers per thread), 8..11 rows in a "tall" CTA of 16 warps (4 per
// sub-partition, 128 registers) for the pairs whose state fits that budget
// and whose per-row shared memory allows it (not Dormand-Prince stages
// 4+5).  The halo warp covers at most 16 rows (two lanes per row for ty + 4
// rows).
constexpr int kPairMaxTY = 7;
constexpr int kPairMaxTYTall = 11;
template <bool TALL>
__host__ __device__ constexpr int pair_threads() {
    return 32 * ((TALL ? kPairMaxTYTall : kPairMaxTY) + 5);
}
__host__ __device__ constexpr int pair_max_ty(int mode) {
    return mode == MODE_PAIR_DOPRI45 ? kPairMaxTY : kPairMaxTYTall;
}


template <typename T>
__host__ __device__ constexpr int pair_vx() {
    return 16 / (int)sizeof(T);
}
// a plane row: 2 halo cells on each side of the 32*VX main cells, the main
// cells starting at a whole vector (column c at OFF + c, OFF = VX)
template <typename T>
__host__ __device__ constexpr int pair_off() {
    return 16 / (int)sizeof(T);
}
template <typename T, int VX>
__host__ __device__ constexpr int pair_pitch() {
    return 2 * pair_off<T>() + 32 * VX;
}
// Y_i: 3 buffers x (ty + 4) rows; Y_{i+1}: 3 buffers x (ty + 2) rows; 2 components
template <typename T, int VX>
__host__ __device__ inline size_t pair_plane_bytes(int ty) {
    return sizeof(T) * 3 * (size_t)((ty + 4) + (ty + 2)) * 2 * pair_pitch<T, VX>();
}
// one ring slot: (ty + 4) rows x NA arrays x 32 lanes of VX-cell vectors,
// then the halo lanes' pairs: NA arrays x 32 lanes x 2 cells
template <typename T, int NK, int VX>
__host__ __device__ inline size_t pair_slot_bytes(int ty) {
    constexpr int NA = 2 * (1 + NK);
    const size_t vec = (size_t)(ty + 4) * NA * 32 * VX * sizeof(T);
    const size_t halo = (size_t)NA * 32 * 2 * sizeof(T);
    return (vec + halo + 127) / 128 * 128;
}
// Values the tile rows' threads keep from phase A to phase C in shared
// memory (thread-private, 3 planes x fields x 2 components): Dormand-Prince
// stages 6+7 the inverse error scale; stages 4+5 the k1..k3 parts of Y6 - u,
// P - u and the error terms, and u (so that Y6 and P add u once, to the
// whole small sum); RK4 stages 3+4 the partial update u + dt (k1/6 + k2/3).
template <int MODE>
__host__ __device__ constexpr int pair_stash_fields() {
    return MODE == MODE_PAIR_DOPRI45 ? 4 : ((MODE == MODE_PAIR_DOPRI67 || MODE == MODE_PAIR_RK4) ? 1 : 0);
}
template <typename T, int MODE, int VX>
__host__ __device__ inline size_t pair_isc_bytes(int ty) {
    return (size_t)pair_stash_fields<MODE>() * 3 * 2 * ty * 32 * VX * sizeof(T);
}
// the input ring starts at a 128-byte boundary of the shared window (+ 128
// bytes of room for that): a warp's 512 contiguous bytes of a slot then
// cover four whole 128-byte lines instead of five
template <typename T, int NK, int MODE, int VX>
__host__ __device__ inline size_t pair_smem_bytes(int ty, int depth) {
    return (pair_plane_bytes<T, VX>(ty) + 15) / 16 * 16 + pair_isc_bytes<T, MODE, VX>(ty) + 128 +
           (size_t)depth * pair_slot_bytes<T, NK, VX>(ty);
}

// Coefficients of one pair launch in T.
template <typename T, int NK>
struct PairCoef {
    T a1[NK > 0 ? NK : 1];  // stage i: Y_i = u + dt sum_j a1_j k_j
    T a2[NK + 1];           // stage i+1: Y_{i+1} = u + dt sum_j a2_j k_j (j <= i)
    T rb[4];                // RK4 update weights of k1..k4
    T dt, ta, tr;
};

template <typename T, int NK>
__device__ __forceinline__ PairCoef<T, NK> pair_coef(const StageArgs& A, double dt, double atol, double rtol) {
    PairCoef<T, NK> C;
#pragma unroll
    for (int j = 0; j < NK; ++j) C.a1[j] = (T)A.a[j];
#pragma unroll
    for (int j = 0; j <= NK; ++j) C.a2[j] = (T)A.bk[j];
    C.rb[0] = (T)A.be[0];
    C.rb[1] = (T)A.be[1];
    C.rb[2] = (T)A.be[2];
    C.rb[3] = (T)A.bf;
    C.dt = (T)dt;
    C.ta = (T)atol;
    C.tr = (T)rtol;
    return C;
}

__device__ __forceinline__ int wrapm(int a, int n) {
    const int m = a % n;
    return m < 0 ? m + n : m;
}

// One segment: column (tx, tyi), output planes [z0, z1).  Called by every
// thread of the CTA (it contains barriers: (z1 - z0) + 4 per segment, the
// same count in the row warps and in the halo warp).
template <typename T, int NK, int MODE, int VX>
__device__ __forceinline__ void pair_segment(const Geom<T>& g, const StagePtrs<T, NK>& P, const PairCoef<T, NK>& C,
                                             T* SA, T* SB, unsigned char* SI, unsigned char* R, int depth, int TY,
                                             int tx, int tyi, int z0, int z1,
                                             typename ErrBits<T>::U& ebits) {
    constexpr int TXW = 32 * VX;
    constexpr int PITCH = pair_pitch<T, VX>();
    constexpr int OFF = pair_off<T>();
    constexpr int NA = 2 * (1 + NK);
    constexpr bool DP = MODE == MODE_PAIR_DOPRI67;
    constexpr bool D45 = MODE == MODE_PAIR_DOPRI45;
    constexpr bool D23 = MODE == MODE_PAIR_DOPRI23;
    constexpr bool RK = MODE == MODE_PAIR_RK4;
    constexpr int NS = pair_stash_fields<MODE>();
    static_assert(!DP || NK == 3, "Dormand-Prince stages 6/7 take Y6, P, the error terms and the inverse scale");
    static_assert(!D45 || NK == 3, "Dormand-Prince stages 4/5 take k1..k3");
    static_assert(!D23 || NK == 1, "Dormand-Prince stages 2/3 take k1");
    static_assert(!RK || NK == 2, "RK4 stages 3/4 take k1, k2");
    using VTy = typename VecT<T, VX>::type;
    using V2 = typename VecT<T, 2>::type;
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int RA = TY + 4, RB = TY + 2;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long plane = (long long)nx * ny;
    const T dt = C.dt;
    // weight of k_i in Y_{i+1} (Dormand-Prince: y5 = P + dt b6 k6) and the
    // stage-6/7 error constants
    const T dta2 = DP ? dt * (T)dp5::B6 : dt * C.a2[NK];
    const T dte6 = dt * (T)dp5::E6, dte7 = dt * (T)dp5::E7;
    // stages 4+5: the k4, k5 weights of Y6, P and the error terms, times dt
    const T d64 = dt * (T)dp5::A64, d65 = dt * (T)dp5::A65;
    const T db4 = dt * (T)dp5::B4, db5 = dt * (T)dp5::B5;
    const T de4 = dt * (T)dp5::E4, de5 = dt * (T)dp5::E5;

    const int x0 = tx * TXW, y0 = tyi * TY;
    const int aw = min(TXW, nx - x0);
    const int ah = min(TY, ny - y0);
    const int nl = aw / VX;
    const bool hw = (w == TY + 4);                  // the halo warp
    const int r = hw ? (lane >> 1) - 2 : w - 2;     // this thread's row, relative to y0
    const int side = lane & 1;                      // halo warp: 0 left, 1 right
    const bool inA = hw ? (lane < 2 * (ah + 4)) : (r < ah + 2 && lane < nl);
    const bool inB = inA && r >= -1 && r < ah + 1;
    const bool inC = !hw && inA && r >= 0 && r < ah;
    const long long rowbase = (long long)nx * wrapm(y0 + r, ny);
    const long long cbase = rowbase + (hw ? (side == 0 ? wrapm(x0 - 2, nx) : wrapm(x0 + aw, nx)) : x0 + VX * lane);
    // halo warp, one cell per lane in the rows (VX = 1, any nx): the pair's
    // second cell wraps on its own and the pair is copied as two cells (an
    // odd nx leaves it 8-byte unaligned)
    const long long cbase1 = rowbase + (side == 0 ? wrapm(x0 - 1, nx) : wrapm(x0 + aw + 1, nx));
    const int col = hw ? (side == 0 ? -2 : aw) : VX * lane;  // shared-memory column of the first cell
    const int hin = side == 0 ? -1 : aw;                      // halo warp: its inner column
    const int hsel = side == 0 ? 1 : 0;                       // ... and its index in the pair

    auto ia = [&](int b, int row, int c, int cx) -> int { return ((b * RA + row + 2) * 2 + c) * PITCH + OFF + cx; };
    auto ib = [&](int b, int row, int c, int cx) -> int { return ((b * RB + row + 1) * 2 + c) * PITCH + OFF + cx; };
    const size_t slot_bytes = pair_slot_bytes<T, NK, VX>(TY);
    const size_t vec_bytes = (size_t)RA * NA * 32 * sizeof(VTy);
    auto rvec = [&](int s, int a) -> VTy* {
        return reinterpret_cast<VTy*>(R + (size_t)s * slot_bytes) + ((size_t)w * NA + a) * 32 + lane;
    };
    // this thread's stash vector of field f, component c in plane buffer k
    // (0..2); tile rows only
    auto siv = [&](int k, int f, int c) -> VTy* {
        return reinterpret_cast<VTy*>(SI) + ((size_t)((k * NS + f) * 2 + c) * TY + r) * 32 + lane;
    };
    auto rhal = [&](int s, int a) -> V2* {
        return reinterpret_cast<V2*>(R + (size_t)s * slot_bytes + vec_bytes) + (size_t)a * 32 + lane;
    };

    // input plane q (z0 - 2 .. z1 + 1) into ring slot s
    auto fetch = [&](int q, int s) {
        if (q <= z1 + 1 && inA) {
            const long long zo = plane * wrapm(q, nz);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
#pragma unroll
                for (int f = 0; f <= NK; ++f) {
                    // stages 6+7: Y6 on every row, P on rows -1..ty, the
                    // error terms and the inverse scale on the tile rows;
                    // RK4 stages 3+4: k1 only on the tile rows (the update)
                    if (DP && f > 0 && !(f == 1 ? inB : inC)) continue;
                    if (RK && f == 1 && !inC) continue;
                    const T* base = (f == 0 ? P.u[c] : P.k[f > 0 ? f - 1 : 0][c]);
                    const T* src = base + cbase + zo;
                    if (hw && VX == 1) {
                        T* dst = reinterpret_cast<T*>(rhal(s, c * (1 + NK) + f));
                        cp_async_vec<sizeof(T)>(dst, src);
                        cp_async_vec<sizeof(T)>(dst + 1, base + cbase1 + zo);
                    } else if (hw)
                        cp_async_vec<2 * sizeof(T)>(rhal(s, c * (1 + NK) + f), src);
                    else
                        cp_async_vec<sizeof(VTy)>(rvec(s, c * (1 + NK) + f), src);
                }
            }
        }
        cp_async_commit();  // one group per plane and thread, empty or not
    };

    // Y_i of NV consecutive cells from the slot (ld(a, v) loads array a) and
    // the second-stage partial P2 = u + dt sum_{j<i} a2_j k_j.  Dormand-Prince
    // stages 6+7 load them (Y6 and P) and, with E (tile rows), the error terms
    // Q and the inverse error scale I.  With E (tile rows), stages 4+5 also
    // form the parts of stage 6's fields that u and k1..k3 give and stages
    // 2+3 the inverse error scale, and hand them, one component at a time,
    // to sink(c, S6, S7, Q, X): S6 = dt (a61 k1 + a62 k2 + a63 k3), S7 = dt
    // (b1 k1 + b3 k3), Q = dt (e1 k1 + e3 k3) (b2 = e2 = 0) and X = u; X = I
    // = 1 / (atol + rtol (|u| + dt |k1|)).  RK4 stages 3+4 with E: I = u + dt
    // (k1/6 + k2/3), the update so far.
    auto formA = [&](auto&& ld, auto& Y, auto& P2, auto& Q, auto& I, auto E, auto&& sink) {
        constexpr int NV = sizeof(Y[0]) / sizeof(T);
        constexpr bool WE = DP && decltype(E)::value;
        constexpr bool W45 = D45 && decltype(E)::value;
        constexpr bool W23 = D23 && decltype(E)::value;
        constexpr bool WR = RK && decltype(E)::value;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (DP) {
                ld(c * (1 + NK), Y[c]);
                ld(c * (1 + NK) + 1, P2[c]);
                if (WE) {
                    ld(c * (1 + NK) + 2, Q[c]);
                    ld(c * (1 + NK) + 3, I[c]);
                }
                continue;
            }
            T uu[NV], s1[NV], s2[NV], k1v[NV], q[NV], s6[NV], s7[NV];
            ld(c * (1 + NK), uu);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                s1[v] = s2[v] = k1v[v] = q[v] = s6[v] = s7[v] = T(0);
            }
#pragma unroll
            for (int j = 0; j < NK; ++j) {
                // RK4 stages 3+4: Y3 = u + dt/2 k2 and Y4 = u + dt k3, so k1
                // enters only the update (tile rows)
                if (RK && j == 0 && !WR) continue;
                T kk[NV];
                ld(c * (1 + NK) + 1 + j, kk);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (RK) {
                        if (j == 1) s1[v] = C.a1[j] * kk[v];
                    } else {
                        s1[v] = (j == 0) ? C.a1[0] * kk[v] : s1[v] + C.a1[j] * kk[v];
                        s2[v] = (j == 0) ? C.a2[0] * kk[v] : s2[v] + C.a2[j] * kk[v];
                    }
                    if (WR) q[v] = (j == 0) ? C.rb[0] * kk[v] : q[v] + C.rb[j] * kk[v];
                    if (W23 && j == 0) k1v[v] = kk[v];
                    if (W45) {
                        if (j == 0) {
                            s6[v] = (T)dp5::A61 * kk[v];
                            s7[v] = (T)dp5::B1 * kk[v];
                            q[v] = (T)dp5::E1 * kk[v];
                        } else if (j == 1) {
                            s6[v] += (T)dp5::A62 * kk[v];
                        } else {
                            s6[v] += (T)dp5::A63 * kk[v];
                            s7[v] += (T)dp5::B3 * kk[v];
                            q[v] += (T)dp5::E3 * kk[v];
                        }
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Y[c][v] = (NK == 0) ? uu[v] : uu[v] + dt * s1[v];
                P2[c][v] = (NK == 0 || RK) ? uu[v] : uu[v] + dt * s2[v];
                if (W45) {
                    s6[v] = dt * s6[v];
                    s7[v] = dt * s7[v];
                    q[v] = dt * q[v];
                }
                if (W23) k1v[v] = ErrBits<T>::recip(C.ta + C.tr * (fabs(uu[v]) + dt * fabs(k1v[v])));
                if (WR) I[c][v] = uu[v] + dt * q[v];
            }
            if (W45) sink(c, s6, s7, q, uu);
            if (W23) sink(c, s6, s7, q, k1v);
        }
    };
    auto nosink = [](int, const T*, const T*, const T*, const T*) {};
    auto react = [&](T yu, T yv, T lu, T lv, T& fu, T& fv) {
        const T uvv = yu * yv * yv;
        fu = g.Du * lu - uvv + g.F * (T(1) - yu);
        fv = g.Dv * lv + uvv - (g.F + g.k) * yv;
    };
    // k = F(Y) (Eq. 2) at this thread's VX cells of a plane: centre Yc and
    // upper z neighbour Yu in registers, the y neighbours and the lower z
    // neighbour from plane buffer S (index function ix; bc: this plane's
    // buffer, bz: the plane below), x neighbours across lanes (xl, xr: the
    // shuffled values of the neighbouring lanes, read from S at the row's
    // ends)
    auto cell_rhs = [&](const T* S, auto&& ix, int bc, int bz, const T(&Yc)[2][VX], const T(&Yu)[2][VX], T xl[2],
                        T xr[2], T(&f)[2][VX]) {
        T lap[2][VX];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (lane == 0) xl[c] = S[ix(bc, r, c, -1)];
            if (lane == nl - 1) xr[c] = S[ix(bc, r, c, aw)];
            T ys[VX], yn[VX], zm[VX];
            lds_v<T, VX>(S + ix(bc, r - 1, c, col), ys);
            lds_v<T, VX>(S + ix(bc, r + 1, c, col), yn);
            lds_v<T, VX>(S + ix(bz, r, c, col), zm);
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                const T xm = (v == 0) ? xl[c] : Yc[c][v - 1];
                const T xp = (v == VX - 1) ? xr[c] : Yc[c][v + 1];
                const T yy = Yc[c][v];
                lap[c][v] = (xm - T(2) * yy + xp) * g.cx + (ys[v] - T(2) * yy + yn[v]) * g.cy +
                            (zm[v] - T(2) * yy + Yu[c][v]) * g.cz;
            }
        }
#pragma unroll
        for (int v = 0; v < VX; ++v) react(Yc[0][v], Yc[1][v], lap[0][v], lap[1][v], f[0][v], f[1][v]);
    };

    for (int i = 0; i < depth; ++i) fetch(z0 - 2 + i, i);
    const int nit = (z1 - z0) + 4;

    // Plane buffers cycle through 3: Y_i of plane q in buffer b = it mod 3,
    // Y_{i+1} of plane q - 1 in buffer b too; so the centre planes of B and C
    // are in buffer b - 1 and their lower z neighbours (own cells) in b - 2.
    if (!hw) {
        // ---------------- row warps ----------------
        // Values carried from one iteration to the next alternate between the
        // X and Y sets (the loop is unrolled twice), so nothing is copied.
        T yaX[2][VX], yaY[2][VX];  // Y_i of plane q (A's output; B's centre one iteration later)
        T ybX[2][VX], ybY[2][VX];  // Y_{i+1} of plane q - 1 (B's output; C's centre one iteration later)
        T p2X[2][VX], p2Y[2][VX];  // P2 (A -> B)
        T qX[2][VX], qY[2][VX];    // Dormand-Prince: Q (A -> B)
        T epX[2][VX], epY[2][VX];  // Dormand-Prince: error through k6 (B -> C)
        T isc[2][VX];              // Dormand-Prince: inverse scale (A -> SI -> C)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                yaX[c][v] = yaY[c][v] = ybX[c][v] = ybY[c][v] = T(0);
                p2X[c][v] = p2Y[c][v] = qX[c][v] = qY[c][v] = epX[c][v] = epY[c][v] = isc[c][v] = T(0);
            }
        // tile-row warps (the longest path: A, B and C every iteration) run
        // the steady state through a copy of the body without run-time phase
        // tests (TILE), so each iteration is one block the compiler can
        // schedule across phases; lanes past the row's end only skip memory
        // accesses there
        const bool act = lane < nl;
        auto body = [&](const bool TILE, int it, int b, int sA, T(&yaN)[2][VX], const T(&yaC)[2][VX], T(&ybN)[2][VX],
                        const T(&ybC)[2][VX], T(&p2N)[2][VX], const T(&p2C)[2][VX], T(&qN)[2][VX],
                        const T(&qC)[2][VX], T(&epN)[2][VX], const T(&epC)[2][VX]) {
            const bool doA = TILE || inA, doB = TILE ? act : (it >= 2 && inB), doC = TILE ? act : (it >= 4 && inC);
            // rows whose error terms (RK4: partial update) are needed
            const bool wide = (DP || D45 || D23 || RK) && (TILE || inC);
            const int q = z0 - 2 + it;
            const int b1 = b == 0 ? 2 : b - 1, b2 = b == 2 ? 0 : b + 1;  // planes q - 1 and q - 2
            // ---- A(q)
            cp_async_wait_pending(depth - 1);
            if (doA) {
                auto ld = [&](int a, T* out) { lds_v<T, VX>(reinterpret_cast<const T*>(rvec(sA, a)), out); };
                // tile rows: stages 4+5 S6, S7, Q and u to the stash;
                // stages 2+3 I straight to its field (no later phase needs it)
                auto sink = [&](int c, const T* s6, const T* s7, const T* qa, const T* ic) {
                    if (!(TILE ? act : true)) return;
                    if (D45) {
                        stv<T, VX>(reinterpret_cast<T*>(siv(b, 0, c)), s6);
                        stv<T, VX>(reinterpret_cast<T*>(siv(b, 1, c)), s7);
                        stv<T, VX>(reinterpret_cast<T*>(siv(b, 2, c)), qa);
                        stv<T, VX>(reinterpret_cast<T*>(siv(b, 3, c)), ic);
                    } else if (q >= z0 && q < z1) {
                        stv<T, VX>(P.o2[c] + cbase + plane * q, ic);
                    }
                };
                if (TILE)
                    formA(ld, yaN, p2N, qN, isc, std::true_type{}, sink);
                else if (wide)
                    formA(ld, yaN, p2N, qN, isc, std::true_type{}, sink);
                else
                    formA(ld, yaN, p2N, qN, isc, std::false_type{}, nosink);
                if (TILE ? act : true) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        stv<T, VX>(SA + ia(b, r, c, col), yaN[c]);
                        if (wide && !D45 && NS > 0) stv<T, VX>(reinterpret_cast<T*>(siv(b, 0, c)), isc[c]);
                    }
                }
            }
            fetch(q + depth, sA);  // the slot's values are in registers: reuse it
            // ---- B(p), p = q - 1: centre yaC, upper z neighbour yaN
            if (TILE || it >= 2) {
                const int p = q - 1;
                T xl[2], xr[2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    xl[c] = __shfl_up_sync(0xffffffffu, yaC[c][VX - 1], 1);
                    xr[c] = __shfl_down_sync(0xffffffffu, yaC[c][0], 1);
                }
                if (doB) {
                    T f[2][VX];
                    cell_rhs(SA, ia, b1, b2, yaC, yaN, xl, xr, f);
                    const bool own = TILE ? p < z1 : (r >= 0 && r < ah && p >= z0 && p < z1);
                    const long long gi = cbase + plane * p;
                    T tu[2][VX] = {};  // RK4: the partial update of plane p (tile rows)
                    if (RK && (TILE || (r >= 0 && r < ah))) {
#pragma unroll
                        for (int c = 0; c < 2; ++c) lds_v<T, VX>(reinterpret_cast<const T*>(siv(b1, 0, c)), tu[c]);
                    }
#pragma unroll
                    for (int c = 0; c < 2; ++c)
#pragma unroll
                        for (int v = 0; v < VX; ++v) {
                            ybN[c][v] = p2C[c][v] + dta2 * f[c][v];
                            if (DP) epN[c][v] = qC[c][v] + dte6 * f[c][v];
                            if (D45) epN[c][v] = f[c][v];  // k4, to phase C
                            if (RK) epN[c][v] = tu[c][v] + dt * C.rb[2] * f[c][v];
                        }
                    if (own && !RK && !D45) {
#pragma unroll
                        for (int c = 0; c < 2; ++c) stv<T, VX>(P.o0[c] + gi, DP ? ybN[c] : f[c]);
                    }
#pragma unroll
                    for (int c = 0; c < 2; ++c) stv<T, VX>(SB + ib(b, r, c, col), ybN[c]);
                }
            }
            // ---- C(o), o = q - 2: centre ybC, upper z neighbour ybN
            if (TILE || it >= 4) {
                const int o = q - 2;
                T xl[2], xr[2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    xl[c] = __shfl_up_sync(0xffffffffu, ybC[c][VX - 1], 1);
                    xr[c] = __shfl_down_sync(0xffffffffu, ybC[c][0], 1);
                }
                if (doC) {
                    T f[2][VX];
                    cell_rhs(SB, ib, b1, b2, ybC, ybN, xl, xr, f);
                    const long long gi = cbase + plane * o;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        if (RK) {
                            T un[VX];
#pragma unroll
                            for (int v = 0; v < VX; ++v) un[v] = epC[c][v] + dt * C.rb[3] * f[c][v];
                            stv<T, VX>(P.o0[c] + gi, un);
                        } else if (D45) {
                            // stage 6's fields: the stashed parts plus the
                            // k4 (epC) and k5 (f) terms
                            T s6[VX], s7[VX], qa[VX], uo[VX];
                            lds_v<T, VX>(reinterpret_cast<const T*>(siv(b2, 0, c)), s6);  // plane q - 2
                            lds_v<T, VX>(reinterpret_cast<const T*>(siv(b2, 1, c)), s7);
                            lds_v<T, VX>(reinterpret_cast<const T*>(siv(b2, 2, c)), qa);
                            lds_v<T, VX>(reinterpret_cast<const T*>(siv(b2, 3, c)), uo);
#pragma unroll
                            for (int v = 0; v < VX; ++v) {
                                const T k4 = epC[c][v], k5 = f[c][v];
                                s6[v] = uo[v] + (d65 * k5 + (d64 * k4 + s6[v]));
                                s7[v] = uo[v] + (db5 * k5 + (db4 * k4 + s7[v]));
                                qa[v] = de5 * k5 + (de4 * k4 + qa[v]);
                            }
                            stv<T, VX>(P.o0[c] + gi, s6);
                            stv<T, VX>(P.o1[c] + gi, s7);
                            stv<T, VX>(P.o2[c] + gi, qa);
                        } else {
                            stv<T, VX>(P.o1[c] + gi, f[c]);
                        }
                        if (DP) {
                            T sc[VX];
                            lds_v<T, VX>(reinterpret_cast<const T*>(siv(b2, 0, c)), sc);  // plane q - 2
#pragma unroll
                            for (int v = 0; v < VX; ++v) {
                                const T err = epC[c][v] + dte7 * f[c][v];
                                ebits = max(ebits, ErrBits<T>::bits(fabs(err) * sc[v]));
                            }
                        }
                    }
                }
            }
            __syncthreads();
        };
        int b = 0, sA = 0;
        auto advance = [&]() {
            b = b == 2 ? 0 : b + 1;
            sA = sA + 1 == depth ? 0 : sA + 1;
        };
        // tile rows: the general body for the first four iterations (phases
        // B and C start at iterations 2 and 4), then the tile body
        const bool tilew = r >= 0 && r < ah;
        const int nit0 = tilew ? 4 : nit;
        int it = 0;
        for (; it < nit0; it += 2) {
            body(false, it, b, sA, yaX, yaY, ybX, ybY, p2X, p2Y, qX, qY, epX, epY);
            advance();
            if (it + 1 < nit0) {
                body(false, it + 1, b, sA, yaY, yaX, ybY, ybX, p2Y, p2X, qY, qX, epY, epX);
                advance();
            }
        }
        if (tilew) {
            for (; it + 1 < nit; it += 2) {
                body(true, it, b, sA, yaX, yaY, ybX, ybY, p2X, p2Y, qX, qY, epX, epY);
                advance();
                body(true, it + 1, b, sA, yaY, yaX, ybY, ybX, p2Y, p2X, qY, qX, epY, epX);
                advance();
            }
            if (it < nit) body(true, it, b, sA, yaX, yaY, ybX, ybY, p2X, p2Y, qX, qY, epX, epY);
        }
    } else {
        // ---------------- halo warp: the inner halo column of its row and side ----------------
        T h0[2] = {T(0), T(0)}, h1[2] = {T(0), T(0)}, h2[2] = {T(0), T(0)};  // Y_i, planes p-1, p, p+1
        T hp2a[2] = {T(0), T(0)}, hp2b[2] = {T(0), T(0)};
        int b = 0, sA = 0;
        for (int it = 0; it < nit; ++it) {
            const int b1 = b == 0 ? 2 : b - 1;
            cp_async_wait_pending(depth - 1);
            if (inA) {
                T Y[2][2], P2[2][2], Qd[2][2], Id[2][2];
                formA(
                    [&](int a, T* out) {
                        const V2 q2 = *rhal(sA, a);
                        out[0] = reinterpret_cast<const T*>(&q2)[0];
                        out[1] = reinterpret_cast<const T*>(&q2)[1];
                    },
                    Y, P2, Qd, Id, std::false_type{}, nosink);
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (VX == 1) {  // the pair's column may be odd
                        SA[ia(b, r, c, col)] = Y[c][0];
                        SA[ia(b, r, c, col) + 1] = Y[c][1];
                    } else {
                        V2 st;
                        reinterpret_cast<T*>(&st)[0] = Y[c][0];
                        reinterpret_cast<T*>(&st)[1] = Y[c][1];
                        *reinterpret_cast<V2*>(SA + ia(b, r, c, col)) = st;
                    }
                    h2[c] = Y[c][hsel];
                    hp2a[c] = P2[c][hsel];
                }
            }
            fetch(z0 - 2 + it + depth, sA);
            if (it >= 2 && inB) {
                T lap[2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const T xm = SA[ia(b1, r, c, hin - 1)];
                    const T xp = SA[ia(b1, r, c, hin + 1)];
                    const T ys = SA[ia(b1, r - 1, c, hin)];
                    const T yn = SA[ia(b1, r + 1, c, hin)];
                    const T yy = h1[c];
                    lap[c] = (xm - T(2) * yy + xp) * g.cx + (ys - T(2) * yy + yn) * g.cy + (h0[c] - T(2) * yy + h2[c]) * g.cz;
                }
                T f[2];
                react(h1[0], h1[1], lap[0], lap[1], f[0], f[1]);
#pragma unroll
                for (int c = 0; c < 2; ++c) SB[ib(b, r, c, hin)] = hp2b[c] + dta2 * f[c];
            }
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                h0[c] = h1[c];
                h1[c] = h2[c];
                hp2b[c] = hp2a[c];
            }
            __syncthreads();
            b = b == 2 ? 0 : b + 1;
            sA = sA + 1 == depth ? 0 : sA + 1;
        }
    }
    cp_async_wait_pending(0);  // no copy may land in the ring after this segment
    __syncthreads();           // the plane buffers are reused by the next segment
}

// CTAs per SM the pair kernel is compiled for: one with 16-byte rows (its
// registers fill the SM at 384 threads), two with one cell per lane
template <int VX>
__host__ __device__ constexpr int pair_min_blocks() {
    return VX == 1 ? 2 : 1;
}

template <typename T, int NK, int MODE, int VX, bool TALL>
__global__ void __launch_bounds__(pair_threads<TALL>(), TALL ? 1 : pair_min_blocks<VX>())
    gs_pair_kernel(const Geom<T> g, const StageArgs A, const int depth) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* SA = reinterpret_cast<T*>(smem_raw);
    T* SB = SA + 3 * (size_t)(A.ty + 4) * 2 * pair_pitch<T, VX>();
    unsigned char* SI = smem_raw + (pair_plane_bytes<T, VX>(A.ty) + 15) / 16 * 16;
    // the ring at the next 128-byte boundary of the shared window (an offset
    // from smem_raw, so the compiler keeps shared-memory addressing)
    unsigned char* R = SI + pair_isc_bytes<T, MODE, VX>(A.ty);
    R += (128u - ((uint32_t)__cvta_generic_to_shared(R) & 127u)) & 127u;
    __shared__ T red[32];
    __shared__ int s_last;

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
    const StagePtrs<T, NK> P = resolve_stage<T, NK, MODE>(A, parity, step, 0);
    const PairCoef<T, NK> C = pair_coef<T, NK>(A, dtd, atol, rtol);
    typename ErrBits<T>::U ebits = 0;
    if (!skip) {
        for_each_segment(A, g.nz, [&](int col, int z0, int z1) {
            pair_segment<T, NK, MODE, VX>(g, P, C, SA, SB, SI, R, depth, A.ty, col % A.ntx, col / A.ntx, z0, z1,
                                          ebits);
        });
    }
    const T emax = ErrBits<T>::value(ebits);
    if ((MODE == MODE_PAIR_DOPRI67 || MODE == MODE_PAIR_RK4) && A.run_ctrl && A.ctrl)
        final_kernel_epilogue<T, MODE>(A, emax, red, &s_last);
}

}  // namespace gsk
