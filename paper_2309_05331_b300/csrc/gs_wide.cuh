// gs_wide.cuh -- vectorised form of the fused Gray-Scott stage kernel for
// grids whose x-extent is a multiple of the vector width VX (FP32: 4 cells =
// 16 bytes or 2 cells = 8 bytes; FP64: 2 cells = 16 bytes).  Same arithmetic contract as gs_stage_kernel (gs_tile.cuh):
//   Y = u + dt sum_j a_j k_j,  f = F(Y),  mode-specific epilogue.
//
// Mapping: a warp owns one row of 32*VX cells (VX cells per lane, one vector
// load per field and component), a CTA owns ty such rows plus one halo row
// above and below (warps 0 and ty+1) and marches over zc planes.  The z
// neighbours of a thread's cells stay in registers (planes z-1, z, z+1); only
// the centre plane goes through shared memory (a 3-buffer ring, one barrier
// per plane) for the y neighbours and the two x-halo columns, which the lanes
// of the two halo warps load.  x neighbours inside the row come from warp
// shuffles.  The stage-7 error terms that do not depend on k7 are folded into
// two numbers per cell when the plane is loaded, so the epilogue of the next
// iteration carries 2 values per cell and component instead of 6.
#pragma once

#include "gs_tile.cuh"

namespace gsk {

// Vector of VX elements of T moved as one access (8 or 16 bytes).
template <typename T, int VX>
struct VecT;
template <>
struct VecT<float, 1> {
    using type = float;
};
template <>
struct VecT<double, 1> {
    using type = double;
};
template <>
struct VecT<float, 4> {
    using type = float4;
};
template <>
struct VecT<float, 2> {
    using type = float2;
};
template <>
struct VecT<double, 2> {
    using type = double2;
};

template <typename T, int VX>
__device__ __forceinline__ void ldv(const T* __restrict__ p, T* out) {
    using VTy = typename VecT<T, VX>::type;
    const VTy q = __ldg(reinterpret_cast<const VTy*>(p));
    const T* qs = reinterpret_cast<const T*>(&q);
#pragma unroll
    for (int v = 0; v < VX; ++v) out[v] = qs[v];
}

template <typename T, int VX>
__device__ __forceinline__ void stv(T* p, const T* v) {
    using VTy = typename VecT<T, VX>::type;
    VTy q;
    T* qs = reinterpret_cast<T*>(&q);
#pragma unroll
    for (int i = 0; i < VX; ++i) qs[i] = v[i];
    *reinterpret_cast<VTy*>(p) = q;
}

// vector shared-memory load (addresses are aligned to the vector by the pitch)
template <typename T, int VX>
__device__ __forceinline__ void lds_v(const T* p, T* out) {
    using VTy = typename VecT<T, VX>::type;
    const VTy q = *reinterpret_cast<const VTy*>(p);
    const T* qs = reinterpret_cast<const T*>(&q);
#pragma unroll
    for (int v = 0; v < VX; ++v) out[v] = qs[v];
}

// Running maximum of the scaled errors as the integer maximum of their bit
// patterns (one instruction per cell).  The ratios are products of two
// non-negative numbers, so they are +0, positive or NaN; for IEEE values
// >= +0 the bit order is the value order, and every NaN pattern (exponent all
// ones, non-zero mantissa, either sign) sorts above +inf, so one NaN ratio
// makes the maximum NaN, as the controller requires.
template <typename T>
struct ErrBits;
template <>
struct ErrBits<float> {
    using U = unsigned;
    static __device__ __forceinline__ U bits(float x) { return __float_as_uint(x); }
    static __device__ __forceinline__ float value(U b) { return __uint_as_float(b); }
    // error scale: a few ulp are irrelevant to the controller
    static __device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
};
template <>
struct ErrBits<double> {
    using U = unsigned long long;
    static __device__ __forceinline__ U bits(double x) { return (U)__double_as_longlong(x); }
    static __device__ __forceinline__ double value(U b) { return __longlong_as_double((long long)b); }
    static __device__ __forceinline__ double recip(double x) { return 1.0 / x; }
};


// row of 32*VX cells + 2 halo columns, padded to a whole vector
template <int VX>
__host__ __device__ constexpr int wide_pitch() {
    return 32 * VX + (VX >= 2 ? VX : 2);
}
template <typename T, int VX>
__host__ __device__ inline size_t wide_smem_bytes(int ty) {
    return sizeof(T) * 3 * (size_t)(ty + 2) * 2 * wide_pitch<VX>();
}

// Per-cell values a final epilogue needs from the plane's inputs.
template <typename T, int NK, int MODE, int VX>
struct Carry {
    // FINAL: u and the stage inputs; DOPRI_FINAL: error scale and folded error terms
    T a[2][VX];
    // DOPRI_S6: a = u + dt sum_{j=1,3,4,5} b_j k_j, b[0] = dt (folded error
    // terms), b[1] = inverse error scale (written as soon as it is formed)
    T b[MODE == MODE_FINAL ? (NK > 0 ? NK : 1) : (MODE == MODE_DOPRI_S6 ? 2 : 1)][2][VX];
};

// Resolved buffers of one stage launch (one grid, or one batched instance).
template <typename T, int NK>
struct StagePtrs {
    const T* u[2];
    const T* k[NK > 0 ? NK : 1][2];
    T* o0[2];
    T* o1[2];
    T* o2[2];
    const T* ex[kMaxNE][2];
};

template <typename T, int NK, int MODE>
__device__ __forceinline__ StagePtrs<T, NK> resolve_stage(const StageArgs& A, int parity, long long step,
                                                          long long off) {
    StagePtrs<T, NK> P;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        P.u[c] = resolve<T>(A.u, c, parity, step) + off;
#pragma unroll
        for (int j = 0; j < NK; ++j) P.k[j][c] = resolve<T>(A.kin[j], c, parity, step) + off;
        P.o0[c] = resolve<T>(A.out0, c, parity, step) + off;
        P.o1[c] = (MODE != MODE_STAGE && A.has_out1) ? resolve<T>(A.out1, c, parity, step) + off : nullptr;
        P.o2[c] = (MODE == MODE_DOPRI_S6 || MODE == MODE_PAIR_DOPRI23 || MODE == MODE_PAIR_DOPRI45)
                      ? resolve<T>(A.out2, c, parity, step) + off
                      : nullptr;
#pragma unroll
        for (int j = 0; j < kMaxNE; ++j)
            P.ex[j][c] = ((MODE == MODE_FINAL || MODE == MODE_DOPRI_S7) && j < A.n_ex)
                             ? resolve<T>(A.ex[j], c, parity, step) + off
                             : nullptr;
    }
    return P;
}

// Scalars of one stage launch: stage coefficients in T, dt and tolerances.
template <typename T, int NK>
struct StageCoef {
    T a[NK > 0 ? NK : 1];
    T bk[NK > 0 ? NK : 1];
    T be[kMaxNE];
    T bf;
    T dt, ta, tr;
    int n_ex, has_out1;
};

template <typename T, int NK>
__device__ __forceinline__ StageCoef<T, NK> stage_coef(const StageArgs& A, double dt, double atol, double rtol) {
    StageCoef<T, NK> C;
#pragma unroll
    for (int j = 0; j < NK; ++j) {
        C.a[j] = (T)A.a[j];
        C.bk[j] = (T)A.bk[j];
    }
#pragma unroll
    for (int j = 0; j < kMaxNE; ++j) C.be[j] = (T)A.be[j];
    C.bf = (T)A.bf;
    C.dt = (T)dt;
    C.ta = (T)atol;
    C.tr = (T)rtol;
    C.n_ex = A.n_ex;
    C.has_out1 = A.has_out1;
    return C;
}

// One segment: column (tx, tyi) of ty rows x 32*VX cells, planes [z0, z1).
// Called by every thread of the CTA (it contains barriers).  Updates emax
// (DOPRI_FINAL) with the scaled errors of this thread's cells.
template <typename T, int NK, int MODE, int VX>
__device__ __forceinline__ void wide_segment(const Geom<T>& g, const StagePtrs<T, NK>& P, const StageCoef<T, NK>& C,
                                             T* S, int TY, int tx, int tyi, int z0, int z1,
                                             typename ErrBits<T>::U& ebits) {
    constexpr int TXW = 32 * VX;
    constexpr int PITCH = wide_pitch<VX>();
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int TYP = TY + 2;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long plane = (long long)nx * ny;
    const T dt = C.dt;
    // Dormand-Prince error weights of k3..k6 (kin = {k1, k3, k4, k5, k6})
    const T ew[4] = {(T)dp5::E3, (T)dp5::E4, (T)dp5::E5, (T)dp5::E6};
    const T e7 = (T)dp5::E7;
    const T dte7 = dt * e7;

    auto sidx = [&](int buf, int ww, int c, int col) -> int { return ((buf * TYP + ww) * 2 + c) * PITCH + col; };

    // Y of VX cells at idx, and the epilogue's per-cell values: the raw
    // inputs (fetch), then the arithmetic on them (form)
    struct Raw {
        T u[2][VX];
        T k[NK > 0 ? NK : 1][2][VX];
    };
    auto fetchY = [&](long long idx, Raw& R) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            ldv<T, VX>(P.u[c] + idx, R.u[c]);
#pragma unroll
            for (int j = 0; j < NK; ++j) ldv<T, VX>(P.k[j][c] + idx, R.k[j][c]);
        }
    };
    auto formY = [&](const Raw& R, T (&Y)[2][VX], Carry<T, NK, MODE, VX>& cr) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const T* uu = R.u[c];
            T s[VX], k1[VX], q[VX];
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                s[v] = T(0);
                q[v] = T(0);
                k1[v] = T(0);
            }
#pragma unroll
            for (int j = 0; j < NK; ++j) {
                const T* kk = R.k[j][c];
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                    s[v] = (j == 0) ? C.a[0] * kk[v] : s[v] + C.a[j] * kk[v];
                    if (MODE == MODE_FINAL) cr.b[j][c][v] = kk[v];
                    if (MODE == MODE_DOPRI_FINAL) {
                        if (j == 0)
                            k1[v] = kk[v];
                        else
                            q[v] += ew[j - 1] * (kk[v] - k1[v]);
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                Y[c][v] = (NK == 0) ? uu[v] : uu[v] + dt * s[v];
                if (MODE == MODE_FINAL) cr.a[c][v] = uu[v];
                if (MODE == MODE_DOPRI_FINAL) {
                    // 1 / (atol + rtol (|u| + dt |k1|)) and dt (sum_{j<7} e_j (k_j - k1) - e7 k1)
                    cr.a[c][v] = ErrBits<T>::recip(C.ta + C.tr * (fabs(uu[v]) + dt * fabs(k1[v])));
                    cr.b[0][c][v] = dt * (q[v] - e7 * k1[v]);
                }
            }
        }
    };
    auto loadY = [&](long long idx, T (&Y)[2][VX], Carry<T, NK, MODE, VX>& cr) {
        Raw R;
        fetchY(idx, R);
        formY(R, Y, cr);
    };
    // Y of one cell (x-halo column)
    auto loadY1 = [&](long long idx, int c) -> T {
        const T uu = __ldg(P.u[c] + idx);
        if (NK == 0) return uu;
        T s = C.a[0] * __ldg(P.k[0][c] + idx);
#pragma unroll
        for (int j = 1; j < NK; ++j) s += C.a[j] * __ldg(P.k[j][c] + idx);
        return uu + dt * s;
    };

    const int x0 = tx * TXW, y0 = tyi * TY;
    const int aw = min(TXW, nx - x0);
    const int nl = (aw + VX - 1) / VX;  // active lanes (aw is a multiple of VX)
    const int ah = min(TY, ny - y0);
    const bool irow = (w >= 1) && (w <= ah);
    const bool act = (w <= ah + 1) && (lane < nl);
    const bool inner = irow && (lane < nl);
    const int y = wrap1(y0 - 1 + w, ny);
    const long long rowb = (long long)nx * y;
    const long long cbase = rowb + x0 + VX * lane;
    // x-halo columns of the interior rows: lane r-1 of the top halo warp
    // takes the left column of row r, of the bottom halo warp the right one
    const bool hwarp = (w == 0) || (w == ah + 1);
    const bool do_halo = hwarp && (lane < ah);
    const int hrow = lane + 1;
    const int hcol = (w == 0) ? TXW : TXW + 1;
    const long long hbase =
        (long long)nx * wrap1(y0 + lane, ny) + ((w == 0) ? wrap1(x0 - 1, nx) : wrap1(x0 + aw, nx));

    T ym[2][VX], yc[2][VX], yp[2][VX];
    Carry<T, NK, MODE, VX> cur, nxt;
    if (inner) loadY(cbase + plane * wrap1(z0 - 1, nz), ym, nxt);
    if (act) {
        loadY(cbase + plane * z0, yc, cur);
#pragma unroll
        for (int c = 0; c < 2; ++c) stv<T, VX>(S + sidx(0, w, c, VX * lane), yc[c]);
    }
    if (do_halo)
        for (int c = 0; c < 2; ++c) S[sidx(0, hrow, c, hcol)] = loadY1(hbase + plane * z0, c);
    // One cell per lane (VX = 1) leaves few bytes in flight per thread, so
    // the row cells' raw inputs of plane z+2 are fetched into registers
    // while plane z is computed and formed one iteration later (PF); wider
    // vectors load plane z+1 in the iteration that needs it.
    constexpr bool PF = VX == 1;
    Raw rn;
    if (PF && act) fetchY(cbase + plane * wrap1(z0 + 1, nz), rn);
    int bz = 0;  // ring buffer of plane z
    for (int z = z0; z < z1; ++z) {
        const int bn = (bz == 2) ? 0 : bz + 1;  // ring buffer of plane z+1
        if (PF) {
            if (act) {
                formY(rn, yp, nxt);
#pragma unroll
                for (int c = 0; c < 2; ++c) stv<T, VX>(S + sidx(bn, w, c, VX * lane), yp[c]);
            }
            if (do_halo)  // two lanes per row: loaded where they are needed
                for (int c = 0; c < 2; ++c) S[sidx(bn, hrow, c, hcol)] = loadY1(hbase + plane * wrap1(z + 1, nz), c);
            if (act && z + 1 < z1)  // plane z+2 is the upper neighbour of the next iteration
                fetchY(cbase + plane * wrap1(z + 2, nz), rn);
        } else {
            const long long zoff = plane * wrap1(z + 1, nz);
            if (act) {
                loadY(cbase + zoff, yp, nxt);
#pragma unroll
                for (int c = 0; c < 2; ++c) stv<T, VX>(S + sidx(bn, w, c, VX * lane), yp[c]);
            }
            if (do_halo)
                for (int c = 0; c < 2; ++c) S[sidx(bn, hrow, c, hcol)] = loadY1(hbase + zoff, c);
        }
        __syncthreads();
        T xl[2], xr[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            xl[c] = __shfl_up_sync(0xffffffffu, yc[c][VX - 1], 1);
            xr[c] = __shfl_down_sync(0xffffffffu, yc[c][0], 1);
        }
        if (inner) {
            T lap[2][VX];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (lane == 0) xl[c] = S[sidx(bz, w, c, TXW)];
                if (lane == nl - 1) xr[c] = S[sidx(bz, w, c, TXW + 1)];
                T ys[VX], yn[VX];
                lds_v<T, VX>(S + sidx(bz, w - 1, c, VX * lane), ys);
                lds_v<T, VX>(S + sidx(bz, w + 1, c, VX * lane), yn);
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                    const T xm = (v == 0) ? xl[c] : yc[c][v - 1];
                    const T xp = (v == VX - 1) ? xr[c] : yc[c][v + 1];
                    const T yy = yc[c][v];
                    lap[c][v] = (xm - T(2) * yy + xp) * g.cx + (ys[v] - T(2) * yy + yn[v]) * g.cy +
                                (ym[c][v] - T(2) * yy + yp[c][v]) * g.cz;
                }
            }
            T f[2][VX];
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                const T uvv = yc[0][v] * yc[1][v] * yc[1][v];
                f[0][v] = g.Du * lap[0][v] - uvv + g.F * (T(1) - yc[0][v]);
                f[1][v] = g.Dv * lap[1][v] + uvv - (g.F + g.k) * yc[1][v];
            }
            const long long i = cbase + plane * z;
            if (MODE == MODE_STAGE) {
                stv<T, VX>(P.o0[0] + i, f[0]);
                stv<T, VX>(P.o0[1] + i, f[1]);
            } else if (MODE == MODE_FINAL) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    T s[VX];
#pragma unroll
                    for (int v = 0; v < VX; ++v) {
                        s[v] = C.bf * f[c][v];
#pragma unroll
                        for (int j = 0; j < NK; ++j) s[v] += C.bk[j] * cur.b[j][c][v];
                    }
#pragma unroll
                    for (int j = 0; j < kMaxNE; ++j) {
                        if (j < C.n_ex) {
                            T e[VX];
                            ldv<T, VX>(P.ex[j][c] + i, e);
#pragma unroll
                            for (int v = 0; v < VX; ++v) s[v] += C.be[j] * e[v];
                        }
                    }
                    T o[VX];
#pragma unroll
                    for (int v = 0; v < VX; ++v) o[v] = cur.a[c][v] + dt * s[v];
                    stv<T, VX>(P.o0[c] + i, o);
                    if (C.has_out1) stv<T, VX>(P.o1[c] + i, f[c]);
                }
            } else {  // MODE_DOPRI_FINAL
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    stv<T, VX>(P.o0[c] + i, yc[c]);
                    stv<T, VX>(P.o1[c] + i, f[c]);
                    if (NK == 5) {
#pragma unroll
                        for (int v = 0; v < VX; ++v) {
                            const T err = cur.b[0][c][v] + dte7 * f[c][v];  // + dt e7 k7
                            ebits = max(ebits, ErrBits<T>::bits(fabs(err) * cur.a[c][v]));
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                ym[c][v] = yc[c][v];
                yc[c][v] = yp[c][v];
            }
        cur = nxt;
        bz = bn;
    }
    __syncthreads();  // the smem ring is reused by the next segment
}

// Last CTA of a final kernel: fold the error maximum into the control
// block, run the controller and set the loop condition.
template <typename T, int MODE>
__device__ __forceinline__ void final_kernel_epilogue(const StageArgs& A, T emax, T* red, int* s_last) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (MODE == MODE_DOPRI_FINAL || MODE == MODE_DOPRI_S7 || MODE == MODE_PAIR_DOPRI67) {
        const T bmax = block_nanmax(emax, red);
        if (tid == 0) atomic_max_nonneg(&A.ctrl->err_bits, (double)bmax);
    }
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&A.ctrl->arrive, 1u);
        *s_last = (prev == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (*s_last && tid == 0) {
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

// The segments (column, planes [z0, z1)) of this CTA.  Column-split schedule
// when A.kper > 0: CTA b owns z-band b / ncols of column b % ncols, so all
// columns sweep the same planes in step; otherwise a balanced linear share of
// the (column, z) space, cut into per-column runs.
template <typename F>
__device__ __forceinline__ void for_each_segment(const StageArgs& A, int nz, F&& body) {
    const int ncols = A.ntx * A.nty;
    if (A.kper > 0) {
        const int col = (int)(blockIdx.x % ncols);
        const int band = (int)(blockIdx.x / ncols);
        const int z0 = (int)((long long)band * nz / A.kper);
        const int z1 = (int)((long long)(band + 1) * nz / A.kper);
        if (band < A.kper && z0 < z1) body(col, z0, z1);
        return;
    }
    const long long L = (long long)ncols * nz;
    const long long s_end = L * (blockIdx.x + 1) / gridDim.x;
    for (long long sg = L * blockIdx.x / gridDim.x; sg < s_end;) {
        const int col = (int)(sg / nz);
        const int z0 = (int)(sg - (long long)col * nz);
        const int z1 = (int)min((long long)nz, z0 + (s_end - sg));
        sg += z1 - z0;
        body(col, z0, z1);
    }
}

template <typename T, int NK, int MODE, int VX>
__global__ void __launch_bounds__(MODE == MODE_STAGE ? 512 : 256) gs_stage_wide_kernel(const Geom<T> g, const StageArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
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
    const StageCoef<T, NK> C = stage_coef<T, NK>(A, dtd, atol, rtol);
    typename ErrBits<T>::U ebits = 0;
    if (!skip) {
        for_each_segment(A, g.nz, [&](int col, int z0, int z1) {
            wide_segment<T, NK, MODE, VX>(g, P, C, S, A.ty, col % A.ntx, col / A.ntx, z0, z1, ebits);
        });
    }
    const T emax = ErrBits<T>::value(ebits);
    if (MODE != MODE_STAGE && A.run_ctrl && A.ctrl) final_kernel_epilogue<T, MODE>(A, emax, red, &s_last);
}

}  // namespace gsk
