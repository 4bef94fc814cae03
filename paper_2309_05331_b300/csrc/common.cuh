// common.cuh -- device-side building blocks shared by the kernels of
// libgs_b300: the on-device control block of an integration, the step-size
// controller, Butcher coefficients, pointer-slot resolution and NaN-aware
// max reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gsk {

// ---------------------------------------------------------------------------
// Butcher coefficients (Table 1).  Dormand-Prince 5(4): rows A[i][j], fifth
// order weights B (= row 7, first same as last), error weights E = B - Bhat
// where Bhat are the embedded fourth-order weights.
// ---------------------------------------------------------------------------
namespace dp5 {
constexpr double A21 = 1.0 / 5;
constexpr double A31 = 3.0 / 40, A32 = 9.0 / 40;
constexpr double A41 = 44.0 / 45, A42 = -56.0 / 15, A43 = 32.0 / 9;
constexpr double A51 = 19372.0 / 6561, A52 = -25360.0 / 2187, A53 = 64448.0 / 6561,
                 A54 = -212.0 / 729;
constexpr double A61 = 9017.0 / 3168, A62 = -355.0 / 33, A63 = 46732.0 / 5247, A64 = 49.0 / 176,
                 A65 = -5103.0 / 18656;
constexpr double B1 = 35.0 / 384, B3 = 500.0 / 1113, B4 = 125.0 / 192, B5 = -2187.0 / 6784,
                 B6 = 11.0 / 84;
// fourth-order embedded weights
constexpr double H1 = 5179.0 / 57600, H3 = 7571.0 / 16695, H4 = 393.0 / 640,
                 H5 = -92097.0 / 339200, H6 = 187.0 / 2100, H7 = 1.0 / 40;
constexpr double E1 = B1 - H1, E3 = B3 - H3, E4 = B4 - H4, E5 = B5 - H5, E6 = B6 - H6,
                 E7 = 0.0 - H7;
}  // namespace dp5

// Controller constants of the adaptive drivers (the paper gives none; this
// library's reading: error order 4, stepper order 5).
constexpr int kMaxConsecutiveRejects = 500;
constexpr long long kMaxAttempts = 10000000LL;

// ---------------------------------------------------------------------------
// On-device control block of one integration call.  Written by the host
// before the call, advanced by the last CTA of each step's final kernel.
// ---------------------------------------------------------------------------
enum CtrlMode : int { CTRL_FIXED = 0, CTRL_ADAPTIVE = 1 };

struct alignas(64) DevCtrl {
    double t;        // current time
    double t0;       // start time of a fixed-step run (t = t0 + step*dt)
    double t_end;    // adaptive end time (may be +inf)
    double dt;       // proposed next step size
    double dt_try;   // size of the step being attempted (after clipping)
    double atol, rtol;
    double last_E;   // norm of the most recent attempt
    unsigned long long err_bits;  // running max of the scaled error (bits of a non-negative double)
    long long n_acc, n_rej, consec, max_acc, n_att, max_att;
    long long step, step_limit;   // fixed-step counter and its end
    double* log_dt;               // optional record of accepted step sizes
    long long log_cap;
    unsigned int arrive;          // CTAs that finished the current final kernel
    int parity;                   // which of two buffers holds the current state
    int status;                   // gs_status of the run
    int done;                     // 1 once the run has ended
    int last;                     // current attempt is clipped to t_end
    int mode;                     // CtrlMode
};

// Bits of a non-negative double order like the double (NaN above +inf).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__device__ __forceinline__ T nanmax(T a, T b) {
    return (isnan(a) || a > b) ? a : b;
}

template <typename T>
__device__ __forceinline__ T warp_nanmax(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide NaN-propagating max; every thread must call it.  red: smem of
// >= 32 elements.  Result valid in every thread after the call.
template <typename T>
__device__ __forceinline__ T block_nanmax(T v, T* red) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    v = warp_nanmax(v);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        T w = (tid < (nthreads + 31) / 32) ? red[tid] : T(0);
        w = warp_nanmax(w);
        if (tid == 0) red[0] = w;
    }
    __syncthreads();
    return red[0];
}

// Step-size controller, run by one thread after the error norm E of the
// attempt (or, in fixed mode, the step) is complete.  Returns 1 if the loop
// must continue.  Implements the adaptive driver documented in gs.h.
__device__ inline int controller_update(DevCtrl* c, double E) {
    if (c->mode == CTRL_FIXED) {
        c->step += 1;
        c->parity ^= 1;
        c->t = c->t0 + (double)c->step * c->dt_try;
        c->done = (c->step >= c->step_limit) ? 1 : 0;
        return !c->done;
    }
    c->n_att += 1;
    c->last_E = E;
    if (!isfinite(E)) {
        c->status = GS_ERR_NONFINITE;
        c->done = 1;
        return 0;
    }
    const double h = c->dt_try;
    if (E > 1.0) {
        c->n_rej += 1;
        c->consec += 1;
        double fac = 0.9 * pow(E, -1.0 / 3.0);
        if (fac < 0.2) fac = 0.2;
        c->dt = h * fac;
        if (c->consec >= kMaxConsecutiveRejects) {
            c->status = GS_ERR_STEP_UNDERFLOW;
            c->done = 1;
            return 0;
        }
    } else {
        c->consec = 0;
        c->parity ^= 1;
        if (c->log_dt && c->n_acc < c->log_cap) c->log_dt[c->n_acc] = h;
        c->n_acc += 1;
        c->t = c->last ? c->t_end : c->t + h;
        if (E < 0.5) {
            double Em = E;
            const double floor5 = 1.0 / 3125.0;  // 5^-5
            if (Em < floor5) Em = floor5;
            c->dt = h * 0.9 * pow(Em, -1.0 / 5.0);
        } else {
            c->dt = h;
        }
    }
    // next attempt, or stop
    if (!(c->t < c->t_end) || (c->max_acc >= 0 && c->n_acc >= c->max_acc)) {
        c->done = 1;
        return 0;
    }
    if (c->n_att >= c->max_att) {
        c->status = GS_ERR_MAX_STEPS;
        c->done = 1;
        return 0;
    }
    double ht = c->dt;
    c->last = 0;
    if (c->t + ht >= c->t_end) {
        ht = c->t_end - c->t;
        c->last = 1;
    }
    if (!(ht > 0.0) || c->t + ht == c->t) {
        c->status = GS_ERR_STEP_UNDERFLOW;
        c->done = 1;
        return 0;
    }
    c->dt_try = ht;
    return 1;
}

// ---------------------------------------------------------------------------
// Pointer slots.  A kernel argument names up to four candidate buffers per
// state component; which one is live is decided on the device from the
// control block, so one captured graph serves every step of a loop:
//   SEL_FIXED : p[0]
//   SEL_CUR   : p[parity]          (current state / current k1)
//   SEL_NEXT  : p[parity ^ 1]      (where the accepted step goes)
//   SEL_RING  : p[(step + off) & 3] (Adams-Bashforth history ring)
// ---------------------------------------------------------------------------
enum SlotSel : int { SEL_FIXED = 0, SEL_CUR = 1, SEL_NEXT = 2, SEL_RING = 3 };

struct Slot {
    void* p[4][2];
    int sel;
    int off;
};

__host__ __device__ inline Slot slot_fixed(void* a0, void* a1) {
    Slot s{};
    s.p[0][0] = a0;
    s.p[0][1] = a1;
    s.sel = SEL_FIXED;
    return s;
}

template <typename T>
__device__ __forceinline__ T* resolve(const Slot& s, int comp, int parity, long long step) {
    int i = 0;
    switch (s.sel) {
        case SEL_CUR: i = parity; break;
        case SEL_NEXT: i = parity ^ 1; break;
        case SEL_RING: i = (int)((step + s.off) & 3); break;
        default: i = 0;
    }
    return reinterpret_cast<T*>(s.p[i][comp]);
}

}  // namespace gsk
