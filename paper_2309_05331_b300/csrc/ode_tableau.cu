// ode_tableau.cu -- the further steppers of Table 1 on ensembles of
// independent scalar ODEs (FP64), with the benchmark families of the
// section "Accuracy Benchmarks": dx/dt = -x, x (1 - x), and the paper's
// exponential family du/dt = c e^t (Eq. 1a, one coefficient c = x y per
// element) and sigmoidal dynamics du/dt = s(t) (1 - s(t)), s = 1 / (1 +
// e^-t) (Eq. 1b).
//
//   - fixed-step explicit Runge-Kutta with any tableau of Table 1 (Euler,
//     modified midpoint, RK4, Dormand-Prince 5, Cash-Karp 5(4), Fehlberg
//     7(8));
//   - Adams-Bashforth with 1..8 steps (Table 1; Fig. 2c,d), the history in
//     registers, started by a one-step method of order >= s (RK4 for s <= 4,
//     the order-8 Fehlberg solution for s >= 5);
//   - Adams-Bashforth-Moulton with 1..8 steps (Table 1): the Adams-Bashforth
//     predictor, one evaluation at the predicted value, the Adams-Moulton
//     corrector (PECE), started like Adams-Bashforth;
//   - error-controlled integration where EVERY element has its own step size
//     and controller (no global norm: the elements are independent), with
//     any embedded pair (Dormand-Prince, Cash-Karp, Fehlberg).
//
// One thread owns one element for the whole call (grid-stride over
// elements): the element is read once and written once, every stage and
// step runs in registers.  The tableaux are compile-time constants, so each
// stage is a chain of FMAs with immediate coefficients and zero entries
// vanish.  Adaptive elements run their own accept/reject loops; a warp
// finishes when its slowest element does.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "gs_internal.h"
#include "tableaux.cuh"
#include "host_util.h"

using namespace gsk;

namespace {

// Adams-Bashforth weights beta_j of f_{m-j} with s steps (published
// rational values: numerators over a common denominator).
__host__ __device__ constexpr double ab_weight(int s, int j) {
    constexpr double n1[1] = {1};
    constexpr double n2[2] = {3, -1};
    constexpr double n3[3] = {23, -16, 5};
    constexpr double n4[4] = {55, -59, 37, -9};
    constexpr double n5[5] = {1901, -2774, 2616, -1274, 251};
    constexpr double n6[6] = {4277, -7923, 9982, -7298, 2877, -475};
    constexpr double n7[7] = {198721, -447288, 705549, -688256, 407139, -134472, 19087};
    constexpr double n8[8] = {434241, -1152169, 2183877, -2664477, 2102243, -1041723, 295767, -36799};
    return s == 1 ? n1[j] : s == 2 ? n2[j] / 2 : s == 3 ? n3[j] / 12 : s == 4 ? n4[j] / 24
         : s == 5 ? n5[j] / 720 : s == 6 ? n6[j] / 1440 : s == 7 ? n7[j] / 60480 : n8[j] / 120960;
}

// The paper's two families depend on x only through a factor of t shared
// by every element: Eq. 1a f = c e^t (g(t) = e^t), Eq. 1b f = s (1 - s),
// s = 1 / (1 + e^-t) (g(t) = f).
template <int KIND>
__host__ __device__ constexpr bool time_only() {
    return KIND == ODE_PAPER_EXP || KIND == ODE_PAPER_SIGMOID;
}
template <int KIND>
__device__ __forceinline__ double gtime(double t) {
    if (KIND == ODE_PAPER_EXP) return exp(t);
    const double s = 1.0 / (1.0 + exp(-t));
    return s * (1.0 - s);
}
// f from g(t) (time_only kinds)
template <int KIND>
__device__ __forceinline__ double frhs_g(double g, double cf) {
    return KIND == ODE_PAPER_EXP ? cf * g : g;
}

// f(t, x) of each family; cf: the element's coefficient (Eq. 1a)
template <int KIND>
__device__ __forceinline__ double frhs(double t, double x, double cf) {
    if (KIND == ODE_EXP_DECAY) return -x;
    if (KIND == ODE_LOGISTIC) return x * (1.0 - x);
    return frhs_g<KIND>(gtime<KIND>(t), cf);
}

// Fixed steps of the time_only kinds evaluate g at the same times for every
// element, so a call first tabulates them: G[m S + i] = g(t_m + c_i dt),
// t_m = t0 + (mlo + m) dt, m < nm, for the S nodes c of tableau TB (S = 1,
// c = 0: the step times).  Times are rounded as the oracle rounds them (the
// product, then the sum); the kernels then read G (one cached load shared by
// a warp) instead of evaluating exponentials per element.
template <int KIND, class TB>
__global__ void __launch_bounds__(256) ode_gtable_kernel(double t0, double dt, long long mlo, long long nm,
                                                         double* __restrict__ G) {
    const long long total = nm * TB::S;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long m = idx / TB::S;
        const int i = (int)(idx - m * TB::S);
        const double tm = __dadd_rn(t0, __dmul_rn((double)(mlo + m), dt));
        G[idx] = gtime<KIND>(__dadd_rn(tm, __dmul_rn(TB::c(i), dt)));
    }
}
// the step times alone (one node, c = 0)
struct TabNode0 {
    static constexpr int S = 1;
    __host__ __device__ static constexpr double c(int) { return 0.0; }
};

// One step of tableau TB: returns the propagated solution; with ERR also
// err = h sum_i (B_i - BH_i) k_i and k1 (for the error scale).
// G: with a table (time_only kinds, fixed steps), g at this step's S stage
// times, else null (g evaluated here)
template <int KIND, class TB, bool ERR>
__device__ __forceinline__ double tab_step(double u, double t, double h, double cf, double& err, double& k1,
                                           const double* __restrict__ G = nullptr) {
    double k[TB::S];
#pragma unroll
    for (int i = 0; i < TB::S; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < i; ++j)
            if (TB::a(i, j) != 0.0) acc += TB::a(i, j) * k[j];
        if (time_only<KIND>() && G)
            k[i] = frhs_g<KIND>(__ldg(G + i), cf);
        else
            k[i] = frhs<KIND>(t + TB::c(i) * h, i == 0 ? u : u + h * acc, cf);
    }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < TB::S; ++i)
        if (TB::b(i) != 0.0) acc += TB::b(i) * k[i];
    if (ERR) {
        double e = 0.0;
#pragma unroll
        for (int i = 0; i < TB::S; ++i)
            if (TB::b(i) - TB::bh(i) != 0.0) e += (TB::b(i) - TB::bh(i)) * k[i];
        err = h * e;
        k1 = k[0];
    }
    return u + h * acc;
}

// G: the time_only kinds' table of g at every stage time (nsteps x TB::S)
template <int KIND, class TB>
__global__ void __launch_bounds__(256) ode_tab_kernel(long long n, double* __restrict__ x,
                                                      const double* __restrict__ coef, double t0, double dt,
                                                      long long nsteps, const double* __restrict__ G) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double u = x[i];
        const double cf = KIND == ODE_PAPER_EXP ? coef[i] : 0.0;
        double e, k1;
        for (long long m = 0; m < nsteps; ++m)
            u = tab_step<KIND, TB, false>(u, t0 + (double)m * dt, dt, cf, e, k1, G ? G + m * TB::S : nullptr);
        x[i] = u;
    }
}

// Adams-Moulton weights of the corrector (node t_{m+1} first), computed on
// the host (am_weights) and passed by value.
struct AmWeights {
    double w[8];
};

// Adams-Bashforth-Moulton with S steps in PECE form: f[j] = f_{m-j} in
// registers; predictor u* = u + dt sum_j ab_j f_{m-j}, f* = f(t_{m+1}, u*),
// corrector u' = u + dt (am_0 f* + sum_{j>=1} am_j f_{m+1-j}).
// Gm, Gs (time_only kinds): g at the step times t_0..t_nsteps and at the
// start-up steps' stage times ((S - 1) x Start::S), else null
template <int KIND, int S>
__global__ void __launch_bounds__(256) ode_abm_kernel(long long n, double* __restrict__ x,
                                                      const double* __restrict__ coef, double t0, double dt,
                                                      long long nsteps, const AmWeights am,
                                                      const double* __restrict__ Gm, const double* __restrict__ Gs) {
    using Start = typename std::conditional<(S <= 4), TabRK4, TabRKF78>::type;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double u = x[i];
        const double cf = KIND == ODE_PAPER_EXP ? coef[i] : 0.0;
        double f[S];
#pragma unroll
        for (int j = 0; j < S; ++j) f[j] = 0.0;
        double e, k1;
        for (long long m = 0; m < nsteps; ++m) {
            const double t = t0 + (double)m * dt;
#pragma unroll
            for (int j = S - 1; j >= 1; --j) f[j] = f[j - 1];
            f[0] = (time_only<KIND>() && Gm) ? frhs_g<KIND>(__ldg(Gm + m), cf) : frhs<KIND>(t, u, cf);
            if (m < S - 1) {
                u = tab_step<KIND, Start, false>(u, t, dt, cf, e, k1, Gs ? Gs + m * Start::S : nullptr);
            } else {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < S; ++j) acc += ab_weight(S, j) * f[j];
                const double fp = (time_only<KIND>() && Gm)
                                      ? frhs_g<KIND>(__ldg(Gm + m + 1), cf)
                                      : frhs<KIND>(t0 + (double)(m + 1) * dt, u + dt * acc, cf);
                double cor = am.w[0] * fp;
#pragma unroll
                for (int j = 1; j < S; ++j) cor += am.w[j] * f[j - 1];
                u = u + dt * cor;
            }
        }
        x[i] = u;
    }
}

// Adams-Bashforth with S steps: f[j] = f_{m-j} in registers.
// Gm, Gs: as for ode_abm_kernel
template <int KIND, int S>
__global__ void __launch_bounds__(256) ode_ab_kernel(long long n, double* __restrict__ x,
                                                     const double* __restrict__ coef, double t0, double dt,
                                                     long long nsteps, const double* __restrict__ Gm,
                                                     const double* __restrict__ Gs) {
    using Start = typename std::conditional<(S <= 4), TabRK4, TabRKF78>::type;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double u = x[i];
        const double cf = KIND == ODE_PAPER_EXP ? coef[i] : 0.0;
        double f[S];
#pragma unroll
        for (int j = 0; j < S; ++j) f[j] = 0.0;
        double e, k1;
        for (long long m = 0; m < nsteps; ++m) {
            const double t = t0 + (double)m * dt;
#pragma unroll
            for (int j = S - 1; j >= 1; --j) f[j] = f[j - 1];
            f[0] = (time_only<KIND>() && Gm) ? frhs_g<KIND>(__ldg(Gm + m), cf) : frhs<KIND>(t, u, cf);
            if (m < S - 1) {
                u = tab_step<KIND, Start, false>(u, t, dt, cf, e, k1, Gs ? Gs + m * Start::S : nullptr);
            } else {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < S; ++j) acc += ab_weight(S, j) * f[j];
                u = u + dt * acc;
            }
        }
        x[i] = u;
    }
}

// Per-element error control: the controller of the adaptive drivers (reject
// E > 1: dt = h max(0.9 E^(-1/(Q-1)), 0.2); accept, and if E < 0.5 grow dt
// = 0.9 h max(E, 5^-P)^(-1/P); clip the last step to t_end) run by each
// element on its own t and dt.  An element stops at t_end, after max_acc
// accepted steps (< 0: no limit), after max_rej consecutive rejections or a
// step that no longer advances t (STEP_UNDERFLOW), on a non-finite error
// (NONFINITE), or after kMaxElementAttempts attempts (MAX_STEPS), which
// bounds the kernel's run time.
//
// Elements need from a few to hundreds of attempts, so a lane that kept one
// element until the slowest lane of its warp finished would idle.  Each warp
// owns a contiguous chunk of the elements instead, and a lane whose element
// has stopped takes the chunk's next one (a ballot; the chunk cursor is the
// same register value in every lane): every loop iteration is one attempt
// of whichever element each lane holds.  An element's arithmetic is the same
// in either order.
constexpr long long kMaxElementAttempts = 1LL << 22;
// bit patterns of 1.0, 0.5 and 0.2 (IEEE binary64)
constexpr long long kBits1 = 0x3FF0000000000000LL, kBitsHalf = 0x3FE0000000000000LL,
                    kBitsFifth = 0x3FC999999999999ALL;

template <int K>
__device__ __forceinline__ double ipow_pos(double y) {  // y^K, K in 1..8, by multiplication
    const double y2 = y * y, y4 = y2 * y2;
    if (K == 1) return y;
    if (K == 2) return y2;
    if (K == 3) return y2 * y;
    if (K == 4) return y4;
    if (K == 5) return y4 * y;
    if (K == 6) return y4 * y2;
    if (K == 7) return y4 * y2 * y;
    return y4 * y4;
}

// The controller's power x^(-1/K), K = KR (a rejection) or KG (growth)
// chosen per lane: an FP32 estimate, then two Newton steps on f(y) = y^-K -
// x in FP64, y <- y ((K + 1) - x y^K) / K, each of which squares the
// relative error (FP32's ~1e-7 -> ~1e-14 -> rounding): a few ulps from the
// exact power, in a small fraction of the FP64 operations of pow.  x > 0
// and finite; beyond FP32's range (a rejection with E > 3e38) the result
// is 0, where the rejection factor is clamped to 0.2 anyway.
template <int KR, int KG>
__device__ __forceinline__ double ctrl_power(double x, bool rej) {
    const double kp1 = rej ? (double)(KR + 1) : (double)(KG + 1);
    const double rk = rej ? 1.0 / (double)KR : 1.0 / (double)KG;
    double y = (double)powf((float)x, rej ? -1.0f / (float)KR : -1.0f / (float)KG);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double yk = rej ? ipow_pos<KR>(y) : ipow_pos<KG>(y);
        y = y * fma(-x, yk, kp1) * rk;
    }
    return y;
}

template <int KIND, class TB>
__global__ void __launch_bounds__(256) ode_adapt_each_kernel(long long n, double* __restrict__ x,
                                                             const double* __restrict__ coef, double t0,
                                                             double t_end, double dt0, double atol, double rtol,
                                                             long long max_acc, long long max_rej,
                                                             double* t_out, double* dt_out, long* na_out,
                                                             long* nr_out, int* st_out) {
    const double grow_floor = pow(5.0, -(double)TB::P);
    const unsigned lane = threadIdx.x & 31u;
    const long long nwarp = (long long)gridDim.x * (blockDim.x / 32);
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const long long chunk = (n + nwarp - 1) / nwarp;
    long long cursor = gw * chunk;                        // next unclaimed element of this warp's chunk
    const long long cend = cursor + chunk < n ? cursor + chunk : n;
    long long i = -1;                                     // element in hand (-1: none)
    double u = 0.0, cf = 0.0, t = 0.0, dt = 0.0;
    long long na = 0, nr = 0, consec = 0, att = 0;
    int st = GS_OK;
    for (;;) {
        const unsigned need = __ballot_sync(0xffffffffu, i < 0 && cursor < cend);
        if (i < 0 && cursor < cend) {
            const long long j = cursor + __popc(need & ((1u << lane) - 1u));
            if (j < cend) {
                i = j;
                u = x[i];
                cf = KIND == ODE_PAPER_EXP ? coef[i] : 0.0;
                t = t0;
                dt = dt0;
                na = nr = consec = att = 0;
                st = GS_OK;
            }
        }
        cursor += __popc(need);
        if (__ballot_sync(0xffffffffu, i >= 0) == 0u) break;  // the chunk is done
        if (i < 0) continue;
        bool fin = false;
        if (!(t < t_end && (max_acc < 0 || na < max_acc))) {
            fin = true;
        } else if (++att > kMaxElementAttempts) {
            st = GS_ERR_MAX_STEPS;
            fin = true;
        } else {
            bool last = false;
            double h = dt;
            if (t + dt >= t_end) {
                h = t_end - t;
                last = true;
            }
            if (!(h > 0.0) || t + h == t) {
                st = GS_ERR_STEP_UNDERFLOW;
                fin = true;
            } else {
                double err, k1;
                const double y = tab_step<KIND, TB, true>(u, t, h, cf, err, k1);
                const double E = fabs(err) / (atol + rtol * (fabs(u) + h * fabs(k1)));
                // E >= 0 (or NaN): the tests and maxima below compare its bit
                // pattern as an integer, which orders non-negative doubles as
                // their values, and leave the FP64 pipe to the arithmetic
                const long long eb = __double_as_longlong(E);
                if (((eb >> 52) & 0x7ff) == 0x7ff) {  // not finite
                    st = GS_ERR_NONFINITE;
                    fin = true;
                } else {
                    // one power for the rejecting and the accepting lanes
                    // alike (its arguments selected per lane), so a warp
                    // holding both does not run it twice; none when every
                    // lane keeps its step (0.5 <= E <= 1, the steady state)
                    const bool rej = eb > kBits1;   // E > 1
                    const bool grow = eb < kBitsHalf;  // E < 0.5
                    double pw = 1.0;
                    if (__any_sync(__activemask(), rej || grow))
                        pw = ctrl_power<TB::Q - 1, TB::P>(
                            rej ? E : __longlong_as_double(max(eb, __double_as_longlong(grow_floor))), rej);
                    if (rej) {
                        ++nr;
                        ++consec;
                        // max(0.9 pw, 0.2), pw >= 0
                        dt = h * __longlong_as_double(max(__double_as_longlong(0.9 * pw), kBitsFifth));
                        if (consec >= max_rej) {
                            st = GS_ERR_STEP_UNDERFLOW;
                            fin = true;
                        }
                    } else {
                        consec = 0;
                        u = y;
                        ++na;
                        t = last ? t_end : t + h;
                        dt = grow ? h * 0.9 * pw : h;
                    }
                }
            }
        }
        if (fin) {
            x[i] = u;
            if (t_out) t_out[i] = t;
            if (dt_out) dt_out[i] = dt;
            if (na_out) na_out[i] = (long)na;
            if (nr_out) nr_out[i] = (long)nr;
            if (st_out) st_out[i] = st;
            i = -1;
        }
    }
}

int sm_count_t() {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return nsm;
}

template <typename K>
int grid_for(K kern, long long n) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0);
    if (occ < 1) occ = 1;
    const long long need = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(need, (long long)sm_count_t() * occ));
}

bool kind_ok(int kind, const double* coef) {
    if (kind == ODE_PAPER_EXP) return coef != nullptr;
    return kind == ODE_EXP_DECAY || kind == ODE_LOGISTIC || kind == ODE_PAPER_SIGMOID;
}

// dispatch over the right-hand side, then the tableau
template <template <int, class> class Launch, class TB, typename... Args>
cudaError_t by_kind(int kind, Args... args) {
    switch (kind) {
        case ODE_EXP_DECAY: return Launch<ODE_EXP_DECAY, TB>::run(args...);
        case ODE_LOGISTIC: return Launch<ODE_LOGISTIC, TB>::run(args...);
        case ODE_PAPER_EXP: return Launch<ODE_PAPER_EXP, TB>::run(args...);
        default: return Launch<ODE_PAPER_SIGMOID, TB>::run(args...);
    }
}
template <template <int, class> class Launch, typename... Args>
cudaError_t by_tab(int method, int kind, Args... args) {
    switch (method) {
        case ODE_TAB_EULER: return by_kind<Launch, TabEuler>(kind, args...);
        case ODE_TAB_RK4: return by_kind<Launch, TabRK4>(kind, args...);
        case ODE_TAB_DOPRI5: return by_kind<Launch, TabDP5>(kind, args...);
        case ODE_TAB_CK54: return by_kind<Launch, TabCK54>(kind, args...);
        case ODE_TAB_MIDPOINT: return by_kind<Launch, TabMidpoint>(kind, args...);
        default: return by_kind<Launch, TabRKF78>(kind, args...);
    }
}

// Stream-ordered table of g for a time_only kind (null for the others):
// nm x TB::S values from step mlo; released with cudaFreeAsync after use.
template <int KIND, class TB>
cudaError_t make_gtable(cudaStream_t s, double t0, double dt, long long mlo, long long nm, double** out) {
    *out = nullptr;
    if (!time_only<KIND>() || nm <= 0) return cudaSuccess;
    const long long total = nm * TB::S;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(out), sizeof(double) * (size_t)total, s);
    if (e != cudaSuccess) {
        *out = nullptr;
        return e;
    }
    const int grid = (int)std::min<long long>((total + 255) / 256, 4096);
    ode_gtable_kernel<KIND, TB><<<grid, 256, 0, s>>>(t0, dt, mlo, nm, *out);
    return cudaGetLastError();
}
void free_gtable(cudaStream_t s, double* G) {
    if (G) cudaFreeAsync(G, s);
}

template <int KIND, class TB>
struct LaunchTab {
    static cudaError_t run(cudaStream_t s, long long n, double* x, const double* coef, double t0, double dt,
                           long long nsteps) {
        double* G = nullptr;
        cudaError_t e = make_gtable<KIND, TB>(s, t0, dt, 0, nsteps, &G);
        if (e == cudaSuccess) {
            auto k = ode_tab_kernel<KIND, TB>;
            k<<<grid_for(k, n), 256, 0, s>>>(n, x, coef, t0, dt, nsteps, G);
            e = cudaGetLastError();
        }
        free_gtable(s, G);
        return e;
    }
};
template <int KIND, class TB>
struct LaunchEach {
    static cudaError_t run(cudaStream_t s, long long n, double* x, const double* coef, double t0, double t_end,
                           double dt0, double atol, double rtol, long long max_acc, long long max_rej,
                           double* t_out, double* dt_out, long* na, long* nr, int* st) {
        auto k = ode_adapt_each_kernel<KIND, TB>;
        k<<<grid_for(k, n), 256, 0, s>>>(n, x, coef, t0, t_end, dt0, atol, rtol, max_acc, max_rej, t_out,
                                           dt_out, na, nr, st);
        return cudaGetLastError();
    }
};

// the tables of the multistep kernels: g at t_0..t_nsteps and at the
// start-up steps' stage times
template <int KIND, int S>
cudaError_t make_ms_tables(cudaStream_t s, double t0, double dt, long long nsteps, double** Gm, double** Gs) {
    using Start = typename std::conditional<(S <= 4), TabRK4, TabRKF78>::type;
    *Gs = nullptr;
    cudaError_t e = make_gtable<KIND, TabNode0>(s, t0, dt, 0, nsteps + 1, Gm);
    if (e == cudaSuccess) e = make_gtable<KIND, Start>(s, t0, dt, 0, std::min<long long>(S - 1, nsteps), Gs);
    return e;
}

template <int KIND, int S>
cudaError_t launch_ab(cudaStream_t s, long long n, double* x, const double* coef, double t0, double dt,
                      long long nsteps) {
    double *Gm = nullptr, *Gs = nullptr;
    cudaError_t e = make_ms_tables<KIND, S>(s, t0, dt, nsteps, &Gm, &Gs);
    if (e == cudaSuccess) {
        auto k = ode_ab_kernel<KIND, S>;
        k<<<grid_for(k, n), 256, 0, s>>>(n, x, coef, t0, dt, nsteps, Gm, Gs);
        e = cudaGetLastError();
    }
    free_gtable(s, Gm);
    free_gtable(s, Gs);
    return e;
}
template <int KIND>
cudaError_t launch_ab_k(int steps, cudaStream_t s, long long n, double* x, const double* coef, double t0,
                        double dt, long long nsteps) {
    switch (steps) {
        case 1: return launch_ab<KIND, 1>(s, n, x, coef, t0, dt, nsteps);
        case 2: return launch_ab<KIND, 2>(s, n, x, coef, t0, dt, nsteps);
        case 3: return launch_ab<KIND, 3>(s, n, x, coef, t0, dt, nsteps);
        case 4: return launch_ab<KIND, 4>(s, n, x, coef, t0, dt, nsteps);
        case 5: return launch_ab<KIND, 5>(s, n, x, coef, t0, dt, nsteps);
        case 6: return launch_ab<KIND, 6>(s, n, x, coef, t0, dt, nsteps);
        case 7: return launch_ab<KIND, 7>(s, n, x, coef, t0, dt, nsteps);
        default: return launch_ab<KIND, 8>(s, n, x, coef, t0, dt, nsteps);
    }
}

// Adams-Moulton weights with s nodes tau_j = 1 - j (j = 0..s-1) on [0, 1]:
// am_j = int_0^1 l_j(tau) dtau, l_j the Lagrange basis polynomial of node j,
// by 8-point Gauss-Legendre quadrature in long double (exact for the
// degree <= 7 integrands; nodes from Newton's method on the Legendre
// recurrence).
AmWeights am_weights(int s) {
    constexpr int Q = 8;
    long double xq[Q], wq[Q];
    for (int q = 0; q < Q; ++q) {
        long double z = cosl(3.14159265358979323846264338327950288L * (q + 0.75L) / (Q + 0.5L));
        long double dp = 1.0L;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1.0L, p1 = z;  // P_0, P_1
            for (int k = 2; k <= Q; ++k) {
                const long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = Q * (z * p1 - p0) / (z * z - 1.0L);  // P_Q'(z)
            const long double dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < 1e-30L) break;
        }
        xq[q] = 0.5L * (1.0L - z);                       // node on [0, 1]
        wq[q] = 1.0L / ((1.0L - z * z) * dp * dp);       // weight on [0, 1] (half of 2 / ((1 - z^2) P'^2))
    }
    AmWeights A{};
    for (int j = 0; j < s; ++j) {
        long double acc = 0.0L;
        for (int q = 0; q < Q; ++q) {
            long double l = 1.0L;
            for (int i = 0; i < s; ++i)
                if (i != j) l *= (xq[q] - (long double)(1 - i)) / (long double)((1 - j) - (1 - i));
            acc += wq[q] * l;
        }
        A.w[j] = (double)acc;
    }
    return A;
}

template <int KIND, int S>
cudaError_t launch_abm(cudaStream_t s, long long n, double* x, const double* coef, double t0, double dt,
                       long long nsteps) {
    double *Gm = nullptr, *Gs = nullptr;
    cudaError_t e = make_ms_tables<KIND, S>(s, t0, dt, nsteps, &Gm, &Gs);
    if (e == cudaSuccess) {
        auto k = ode_abm_kernel<KIND, S>;
        k<<<grid_for(k, n), 256, 0, s>>>(n, x, coef, t0, dt, nsteps, am_weights(S), Gm, Gs);
        e = cudaGetLastError();
    }
    free_gtable(s, Gm);
    free_gtable(s, Gs);
    return e;
}
template <int KIND>
cudaError_t launch_abm_k(int steps, cudaStream_t s, long long n, double* x, const double* coef, double t0,
                         double dt, long long nsteps) {
    switch (steps) {
        case 1: return launch_abm<KIND, 1>(s, n, x, coef, t0, dt, nsteps);
        case 2: return launch_abm<KIND, 2>(s, n, x, coef, t0, dt, nsteps);
        case 3: return launch_abm<KIND, 3>(s, n, x, coef, t0, dt, nsteps);
        case 4: return launch_abm<KIND, 4>(s, n, x, coef, t0, dt, nsteps);
        case 5: return launch_abm<KIND, 5>(s, n, x, coef, t0, dt, nsteps);
        case 6: return launch_abm<KIND, 6>(s, n, x, coef, t0, dt, nsteps);
        case 7: return launch_abm<KIND, 7>(s, n, x, coef, t0, dt, nsteps);
        default: return launch_abm<KIND, 8>(s, n, x, coef, t0, dt, nsteps);
    }
}

}  // namespace

extern "C" {

gs_status ode_integrate_tableau(ode_rhs kind, ode_tableau method, long n, double* x, const double* coef,
                                double t0, double dt, long nsteps, void* stream) {
    if (!kind_ok(kind, coef) || method < ODE_TAB_EULER || method > ODE_TAB_MIDPOINT || n < 0 || nsteps < 0 ||
        !std::isfinite(dt) || !std::isfinite(t0))
        return GS_ERR_INVALID;
    if (n > 0 && !x) return GS_ERR_INVALID;
    if (n == 0 || nsteps == 0) return GS_OK;
    const cudaError_t e = by_tab<LaunchTab>(method, kind, (cudaStream_t)stream, (long long)n, x, coef, t0, dt,
                                            (long long)nsteps);
    if (e != cudaSuccess) {
        set_global_error(e, "ode_integrate_tableau");
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

gs_status ode_integrate_ab_steps(ode_rhs kind, int steps, long n, double* x, const double* coef, double t0,
                                 double dt, long nsteps, void* stream) {
    if (!kind_ok(kind, coef) || steps < 1 || steps > 8 || n < 0 || nsteps < 0 || !std::isfinite(dt) ||
        !std::isfinite(t0))
        return GS_ERR_INVALID;
    if (n > 0 && !x) return GS_ERR_INVALID;
    if (n == 0 || nsteps == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    switch (kind) {
        case ODE_EXP_DECAY: e = launch_ab_k<ODE_EXP_DECAY>(steps, s, n, x, coef, t0, dt, nsteps); break;
        case ODE_LOGISTIC: e = launch_ab_k<ODE_LOGISTIC>(steps, s, n, x, coef, t0, dt, nsteps); break;
        case ODE_PAPER_EXP: e = launch_ab_k<ODE_PAPER_EXP>(steps, s, n, x, coef, t0, dt, nsteps); break;
        default: e = launch_ab_k<ODE_PAPER_SIGMOID>(steps, s, n, x, coef, t0, dt, nsteps);
    }
    if (e != cudaSuccess) {
        set_global_error(e, "ode_integrate_ab_steps");
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

gs_status ode_integrate_abm_steps(ode_rhs kind, int steps, long n, double* x, const double* coef, double t0,
                                  double dt, long nsteps, void* stream) {
    if (!kind_ok(kind, coef) || steps < 1 || steps > 8 || n < 0 || nsteps < 0 || !std::isfinite(dt) ||
        !std::isfinite(t0))
        return GS_ERR_INVALID;
    if (n > 0 && !x) return GS_ERR_INVALID;
    if (n == 0 || nsteps == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    switch (kind) {
        case ODE_EXP_DECAY: e = launch_abm_k<ODE_EXP_DECAY>(steps, s, n, x, coef, t0, dt, nsteps); break;
        case ODE_LOGISTIC: e = launch_abm_k<ODE_LOGISTIC>(steps, s, n, x, coef, t0, dt, nsteps); break;
        case ODE_PAPER_EXP: e = launch_abm_k<ODE_PAPER_EXP>(steps, s, n, x, coef, t0, dt, nsteps); break;
        default: e = launch_abm_k<ODE_PAPER_SIGMOID>(steps, s, n, x, coef, t0, dt, nsteps);
    }
    if (e != cudaSuccess) {
        set_global_error(e, "ode_integrate_abm_steps");
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

gs_status ode_am_weights(int steps, double* w) {
    if (steps < 1 || steps > 8 || !w) return GS_ERR_INVALID;
    const AmWeights A = am_weights(steps);
    for (int j = 0; j < steps; ++j) w[j] = A.w[j];
    return GS_OK;
}

gs_status ode_integrate_adaptive_each(ode_rhs kind, ode_tableau method, long n, double* x, const double* coef,
                                      double t0, double t_end, double dt0, double atol, double rtol,
                                      long max_acc, long max_rej, double* t_out, double* dt_out, long* n_acc,
                                      long* n_rej, int* status, void* stream) {
    if (!kind_ok(kind, coef) ||
        (method != ODE_TAB_DOPRI5 && method != ODE_TAB_CK54 && method != ODE_TAB_RKF78) || n < 0 ||
        !std::isfinite(t0) || !std::isfinite(t_end) || !(dt0 > 0.0) || !std::isfinite(dt0) || !(atol >= 0.0) ||
        !(rtol >= 0.0) || !(atol + rtol > 0.0) || max_rej < 1)
        return GS_ERR_INVALID;
    if (n > 0 && !x) return GS_ERR_INVALID;
    if (n == 0) return GS_OK;
    const cudaError_t e = by_tab<LaunchEach>(method, kind, (cudaStream_t)stream, (long long)n, x, coef, t0, t_end,
                                             dt0, atol, rtol, (long long)max_acc, (long long)max_rej, t_out, dt_out,
                                             n_acc, n_rej, status);
    if (e != cudaSuccess) {
        set_global_error(e, "ode_integrate_adaptive_each");
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

}  // extern "C"
