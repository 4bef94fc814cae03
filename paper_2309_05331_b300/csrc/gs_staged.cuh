// gs_staged.cuh -- staged form of the vectorised Gray-Scott stage kernel.
//
// Same arithmetic and the same thread mapping as gs_stage_wide_kernel
// (gs_wide.cuh): a warp owns a row of 32*VX cells (one 16-byte vector per
// lane), a CTA owns ty rows plus a halo row above and below, the z
// neighbours stay in registers and the centre plane of Y goes through a
// 3-buffer shared ring with one barrier per plane.
//
// What differs is how the inputs arrive.  The wide form loads plane z+1 from
// global memory at the top of iteration z and waits for it, so every plane
// exposes one full DRAM latency and the loads occupy registers.  Here each
// thread copies its own input vectors (u and the stage inputs k_j, both
// components) with cp.async into a per-thread slot of a shared-memory ring
// DEPTH planes ahead of the plane it forms Y for; lanes of the two halo warps
// do the same for the x-halo columns with 4- or 8-byte copies.  A slot is
// written and read only by the thread that issued its copies, so
// cp.async.wait_group (a hardware wait, no polling) is the only ordering the
// ring needs.  While plane z is computed, DEPTH planes of inputs are in
// flight per thread, without holding registers.
//
// Plane q (counted from z0 - 1, the lower z neighbour of the first plane)
// lives in slot (q - z0 + 1) % DEPTH.  Iteration z waits for plane z+1,
// forms Y(z+1) from it, then reuses the slot for plane z+1+DEPTH.
#pragma once

#include "gs_wide.cuh"

namespace gsk {

constexpr int kMaxDepth = 3;
constexpr size_t kMaxSmemPerCta = 227 * 1024;  // opt-in dynamic shared memory per CTA

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
// one vector of BYTES (4, 8: through L1; 16: L2 only)
template <int BYTES>
__device__ __forceinline__ void cp_async_vec(void* smem, const void* gmem) {
    if constexpr (BYTES == 16)
        cp_async16(smem, gmem);
    else
        cp_async_small<BYTES>(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most n of this thread's committed groups are pending (n < kMaxDepth)
__device__ __forceinline__ void cp_async_wait_pending(int n) {
    if (n <= 0)
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    else if (n == 1)
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else
        asm volatile("cp.async.wait_group 2;\n" ::: "memory");
}

// Shared-memory layout of one launch: the Y ring of the wide form, then DEPTH
// raw slots.  A slot holds (ty+2) rows x NA arrays x 32 lanes of 16-byte
// vectors, then the x-halo columns: 2 sides x NA arrays x ty rows of T.
// Arrays of a slot: u and k_1..k_NK (two components each), then NP
// pointwise arrays (split stage 7: error terms and inverse scale, two
// components each; copied for the tile's own rows only).
template <int MODE>
__host__ __device__ constexpr int staged_pointwise() {
    return MODE == MODE_DOPRI_S7 ? 4 : 0;
}
template <typename T, int NK, int VX, int NP = 0>
__host__ __device__ constexpr int staged_arrays() {
    return 2 * (1 + NK) + NP;
}
template <typename T, int NK, int VX, int NP = 0>
__host__ __device__ inline size_t staged_slot_bytes(int ty) {
    const size_t vec = (size_t)(ty + 2) * staged_arrays<T, NK, VX, NP>() * 32 * sizeof(T) * VX;
    const size_t halo = (size_t)2 * staged_arrays<T, NK, VX, NP>() * ty * sizeof(T);
    return (vec + halo + 15) / 16 * 16;
}
template <typename T, int NK, int VX, int NP = 0>
__host__ __device__ inline size_t staged_smem_bytes(int ty, int depth) {
    return (wide_smem_bytes<T, VX>(ty) + 15) / 16 * 16 + (size_t)depth * staged_slot_bytes<T, NK, VX, NP>(ty);
}

template <typename T, int NK, int MODE, int VX>
__device__ __forceinline__ void staged_segment(const Geom<T>& g, const StagePtrs<T, NK>& P, const StageCoef<T, NK>& C,
                                               T* S, unsigned char* R, int depth, int TY, int tx, int tyi, int z0,
                                               int z1, typename ErrBits<T>::U& ebits) {
    static_assert(sizeof(T) * VX == 4 || sizeof(T) * VX == 8 || sizeof(T) * VX == 16, "4-, 8- or 16-byte vectors");
    constexpr int TXW = 32 * VX;
    constexpr int PITCH = wide_pitch<VX>();
    constexpr int NP = staged_pointwise<MODE>();
    constexpr int NA = staged_arrays<T, NK, VX, NP>();
    using VTy = typename VecT<T, VX>::type;
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int TYP = TY + 2;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long plane = (long long)nx * ny;
    const T dt = C.dt;
    const T ew[4] = {(T)dp5::E3, (T)dp5::E4, (T)dp5::E5, (T)dp5::E6};
    const T e7 = (T)dp5::E7;
    const T dte7 = dt * e7;
    // stage 6 of the split scheme: b of k1, k3, k4, k5; e3..e5 are ew[0..2]
    const T bw[4] = {(T)dp5::B1, (T)dp5::B3, (T)dp5::B4, (T)dp5::B5};
    const T e67 = (T)(dp5::E6 + dp5::E7), dtb6 = dt * (T)dp5::B6, dte6 = dt * (T)dp5::E6;
    const size_t slot_bytes = staged_slot_bytes<T, NK, VX, NP>(TY);
    const size_t vec_bytes = (size_t)TYP * NA * 32 * sizeof(VTy);

    auto sidx = [&](int buf, int ww, int c, int col) -> int { return ((buf * TYP + ww) * 2 + c) * PITCH + col; };
    // this thread's vector of array a in slot s; array a = c * (1 + NK) + f, f = 0: u, f = 1 + j: k_j
    auto rvec = [&](int s, int a) -> VTy* {
        return reinterpret_cast<VTy*>(R + (size_t)s * slot_bytes) + ((size_t)w * NA + a) * 32 + lane;
    };
    auto rhalo = [&](int s, int side, int a, int row) -> T* {
        return reinterpret_cast<T*>(R + (size_t)s * slot_bytes + vec_bytes) + ((size_t)side * NA + a) * TY + row;
    };

    const int x0 = tx * TXW, y0 = tyi * TY;
    const int aw = min(TXW, nx - x0);
    const int nl = (aw + VX - 1) / VX;
    const int ah = min(TY, ny - y0);
    const bool irow = (w >= 1) && (w <= ah);
    const bool act = (w <= ah + 1) && (lane < nl);
    const bool inner = irow && (lane < nl);
    const int y = wrap1(y0 - 1 + w, ny);
    const long long cbase = (long long)nx * y + x0 + VX * lane;
    const bool hwarp = (w == 0) || (w == ah + 1);
    const bool do_halo = hwarp && (lane < ah);
    const int side = (w == 0) ? 0 : 1;
    const int hrow = lane + 1;
    const int hcol = TXW + side;
    const long long hbase =
        (long long)nx * wrap1(y0 + lane, ny) + ((w == 0) ? wrap1(x0 - 1, nx) : wrap1(x0 + aw, nx));

    // copies of plane q (q = z0 - 1 .. z1) into its slot; planes past z1 are not needed
    auto fetch = [&](int q) {
        if (q <= z1) {
            const int s = (q - z0 + 1) % depth;
            const long long zo = plane * (q < 0 ? q + nz : (q >= nz ? q - nz : q));
            if (act) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    cp_async_vec<sizeof(VTy)>(rvec(s, c * (1 + NK)), P.u[c] + cbase + zo);
#pragma unroll
                    for (int j = 0; j < NK; ++j)
                        cp_async_vec<sizeof(VTy)>(rvec(s, c * (1 + NK) + 1 + j), P.k[j][c] + cbase + zo);
                }
            }
            if (NP > 0 && inner) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    cp_async_vec<sizeof(VTy)>(rvec(s, 2 * (1 + NK) + c), P.ex[0][c] + cbase + zo);
                    cp_async_vec<sizeof(VTy)>(rvec(s, 2 * (1 + NK) + 2 + c), P.ex[1][c] + cbase + zo);
                }
            }
            if (do_halo) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    cp_async_small<sizeof(T)>(rhalo(s, side, c * (1 + NK), lane), P.u[c] + hbase + zo);
#pragma unroll
                    for (int j = 0; j < NK; ++j)
                        cp_async_small<sizeof(T)>(rhalo(s, side, c * (1 + NK) + 1 + j, lane), P.k[j][c] + hbase + zo);
                }
            }
        }
        cp_async_commit();  // every thread commits one group per plane, empty or not
    };

    // Y of this thread's VX cells from slot s, and the epilogue's per-cell values
    auto formY = [&](int s, T (&Y)[2][VX], Carry<T, NK, MODE, VX>& cr) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            T uu[VX];
            lds_v<T, VX>(reinterpret_cast<const T*>(rvec(s, c * (1 + NK))), uu);
            T sacc[VX], k1[VX], q[VX], sb[VX], pe[VX], pi[VX];
            if (NP > 0) {
                lds_v<T, VX>(reinterpret_cast<const T*>(rvec(s, 2 * (1 + NK) + c)), pe);
                lds_v<T, VX>(reinterpret_cast<const T*>(rvec(s, 2 * (1 + NK) + 2 + c)), pi);
            }
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                sacc[v] = T(0);
                q[v] = T(0);
                k1[v] = T(0);
                sb[v] = T(0);
            }
#pragma unroll
            for (int j = 0; j < NK; ++j) {
                T kk[VX];
                lds_v<T, VX>(reinterpret_cast<const T*>(rvec(s, c * (1 + NK) + 1 + j)), kk);
#pragma unroll
                for (int v = 0; v < VX; ++v) {
                    sacc[v] = (j == 0) ? C.a[0] * kk[v] : sacc[v] + C.a[j] * kk[v];
                    if (MODE == MODE_FINAL) cr.b[j][c][v] = kk[v];
                    if (MODE == MODE_DOPRI_FINAL) {
                        if (j == 0)
                            k1[v] = kk[v];
                        else
                            q[v] += ew[j - 1] * (kk[v] - k1[v]);
                    }
                    if (MODE == MODE_DOPRI_S6) {
                        // inputs k1..k5; b2 = e2 = 0
                        if (j == 0) {
                            k1[v] = kk[v];
                            sb[v] = bw[0] * kk[v];
                        } else if (j >= 2) {
                            sb[v] += bw[j - 1] * kk[v];
                            q[v] += ew[j - 2] * (kk[v] - k1[v]);
                        }
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                Y[c][v] = (NK == 0) ? uu[v] : uu[v] + dt * sacc[v];
                if (MODE == MODE_FINAL) cr.a[c][v] = uu[v];
                if (MODE == MODE_DOPRI_FINAL) {
                    // 1 / (atol + rtol (|u| + dt |k1|)) and dt (sum_{j<7} e_j (k_j - k1) - e7 k1)
                    cr.a[c][v] = ErrBits<T>::recip(C.ta + C.tr * (fabs(uu[v]) + dt * fabs(k1[v])));
                    cr.b[0][c][v] = dt * (q[v] - e7 * k1[v]);
                }
                if (MODE == MODE_DOPRI_S7) {  // error terms and inverse scale of stage 6
                    cr.b[0][c][v] = pe[v];
                    cr.a[c][v] = pi[v];
                }
                if (MODE == MODE_DOPRI_S6) {
                    // u + dt sum_{j=1,3,4,5} b_j k_j, dt (sum_{j=3,4,5} e_j (k_j - k1) - (e6 + e7) k1),
                    // 1 / (atol + rtol (|u| + dt |k1|))
                    cr.a[c][v] = uu[v] + dt * sb[v];
                    cr.b[0][c][v] = dt * (q[v] - e67 * k1[v]);
                    cr.b[1][c][v] = ErrBits<T>::recip(C.ta + C.tr * (fabs(uu[v]) + dt * fabs(k1[v])));
                }
            }
        }
    };
    // Y of the x-halo cell of this lane's row, from slot s
    auto formY1 = [&](int s, int c) -> T {
        const T uu = *rhalo(s, side, c * (1 + NK), lane);
        if (NK == 0) return uu;
        T sacc = C.a[0] * *rhalo(s, side, c * (1 + NK) + 1, lane);
#pragma unroll
        for (int j = 1; j < NK; ++j) sacc += C.a[j] * *rhalo(s, side, c * (1 + NK) + 1 + j, lane);
        return uu + dt * sacc;
    };

    // prologue: planes z0 - 1 .. z0 - 2 + depth in flight
    for (int i = 0; i < depth; ++i) fetch(z0 - 1 + i);
    T ym[2][VX], yc[2][VX], yp[2][VX];
    Carry<T, NK, MODE, VX> cur, nxt;
    cp_async_wait_pending(depth - 1);  // plane z0 - 1
    if (inner) formY(0, ym, nxt);
    fetch(z0 - 1 + depth);
    cp_async_wait_pending(depth - 1);  // plane z0
    // split stage 6: the inverse error scale of a plane is written as soon as
    // the plane is formed (its own rows only)
    auto put_isc = [&](int zz, const Carry<T, NK, MODE, VX>& cr) {
        if (MODE == MODE_DOPRI_S6 && inner) {
            const long long i = cbase + plane * zz;
#pragma unroll
            for (int c = 0; c < 2; ++c) stv<T, VX>(P.o2[c] + i, cr.b[MODE == MODE_DOPRI_S6 ? 1 : 0][c]);
        }
    };
    {
        const int s = 1 % depth;
        if (act) {
            formY(s, yc, cur);
#pragma unroll
            for (int c = 0; c < 2; ++c) stv<T, VX>(S + sidx(0, w, c, VX * lane), yc[c]);
            put_isc(z0, cur);
        }
        if (do_halo)
            for (int c = 0; c < 2; ++c) S[sidx(0, hrow, c, hcol)] = formY1(s, c);
    }
    fetch(z0 + depth);
    int bz = 0;
    for (int z = z0; z < z1; ++z) {
        const int bn = (bz == 2) ? 0 : bz + 1;
        const int s = (z + 2 - z0) % depth;  // slot of plane z + 1
        cp_async_wait_pending(depth - 1);
        if (act) {
            formY(s, yp, nxt);
#pragma unroll
            for (int c = 0; c < 2; ++c) stv<T, VX>(S + sidx(bn, w, c, VX * lane), yp[c]);
            if (z + 1 < z1) put_isc(z + 1, nxt);
        }
        if (do_halo)
            for (int c = 0; c < 2; ++c) S[sidx(bn, hrow, c, hcol)] = formY1(s, c);
        // the slot's values are in registers (and stored above): reuse it
        fetch(z + 1 + depth);
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
                    T sacc[VX];
#pragma unroll
                    for (int v = 0; v < VX; ++v) {
                        sacc[v] = C.bf * f[c][v];
#pragma unroll
                        for (int j = 0; j < NK; ++j) sacc[v] += C.bk[j] * cur.b[j][c][v];
                    }
#pragma unroll
                    for (int j = 0; j < kMaxNE; ++j) {
                        if (j < C.n_ex) {
                            T e[VX];
                            ldv<T, VX>(P.ex[j][c] + i, e);
#pragma unroll
                            for (int v = 0; v < VX; ++v) sacc[v] += C.be[j] * e[v];
                        }
                    }
                    T o[VX];
#pragma unroll
                    for (int v = 0; v < VX; ++v) o[v] = cur.a[c][v] + dt * sacc[v];
                    stv<T, VX>(P.o0[c] + i, o);
                    if (C.has_out1) stv<T, VX>(P.o1[c] + i, f[c]);
                }
            } else if (MODE == MODE_DOPRI_S6) {
                // k6 = f: y5 = (u + dt sum_{j<6} b_j k_j) + dt b6 k6, error terms up to k6
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    T y5[VX], ep[VX];
#pragma unroll
                    for (int v = 0; v < VX; ++v) {
                        y5[v] = cur.a[c][v] + dtb6 * f[c][v];
                        ep[v] = cur.b[0][c][v] + dte6 * f[c][v];
                    }
                    stv<T, VX>(P.o0[c] + i, y5);
                    stv<T, VX>(P.o1[c] + i, ep);
                }
            } else if (MODE == MODE_DOPRI_S7) {
                // k7 = F(y5); error = stage-6 terms + dt e7 k7, scaled
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    stv<T, VX>(P.o0[c] + i, f[c]);
#pragma unroll
                    for (int v = 0; v < VX; ++v) {
                        const T err = cur.b[0][c][v] + dte7 * f[c][v];
                        ebits = max(ebits, ErrBits<T>::bits(fabs(err) * cur.a[c][v]));
                    }
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
    cp_async_wait_pending(0);  // no copy may land in the ring after this segment
    __syncthreads();           // the Y ring is reused by the next segment
}

// Every mode takes tiles of up to kMaxTY rows (512 threads): the final
// kernels keep no stage inputs in flight in registers here, so they fit the
// 128 registers a 512-thread CTA allows.
// Every mode takes tiles of up to kMaxTY rows (512 threads): with no input
// in flight in registers, even the final kernels fit the 128 registers a
// 512-thread CTA allows.  (A tighter bound that buys more resident CTAs was
// measured slower: the kernel wants the registers more than the warps.)
template <typename T, int NK, int MODE, int VX>
__global__ void __launch_bounds__(512) gs_stage_staged_kernel(const Geom<T> g, const StageArgs A, const int depth) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    unsigned char* R = smem_raw + (wide_smem_bytes<T, VX>(A.ty) + 15) / 16 * 16;
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
            staged_segment<T, NK, MODE, VX>(g, P, C, S, R, depth, A.ty, col % A.ntx, col / A.ntx, z0, z1, ebits);
        });
    }
    const T emax = ErrBits<T>::value(ebits);
    if (MODE != MODE_STAGE && A.run_ctrl && A.ctrl) final_kernel_epilogue<T, MODE>(A, emax, red, &s_last);
}

}  // namespace gsk
