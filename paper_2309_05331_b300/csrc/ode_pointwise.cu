// ode_pointwise.cu -- explicit steppers for ensembles of independent scalar
// ODEs dx_i/dt = f(x_i) in FP64 (the exponential and sigmoidal benchmark
// dynamics of the section "Accuracy Benchmarks", in their autonomous forms
// dx/dt = -x and dx/dt = x (1 - x)).
//
// Fixed-step methods need no communication between elements, so all steps of
// an element run in registers inside one kernel: x is read once and written
// once per call.  The error-controlled Dormand-Prince driver keeps ONE step
// size for the whole vector (one state with a global norm, section
// "Architecture and nomenclature of Boost Odeint"), so every attempt ends with
// a grid-wide max-reduction; one kernel per attempt, the controller runs in
// the last CTA and drives a CUDA-graph WHILE loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "host_util.h"

using namespace gsk;

namespace {

template <int KIND>
__device__ __forceinline__ double rhs(double x) {
    if (KIND == ODE_EXP_DECAY) return -x;
    return x * (1.0 - x);
}

// One Dormand-Prince 5(4) attempt of element x with step h: returns y5, the
// error magnitude |err| and its scale atol + rtol (|x| + h |k1|).
template <int KIND>
__device__ __forceinline__ double dp5_attempt(double x, double h, double atol, double rtol, double& aerr,
                                              double& scale) {
    using namespace dp5;
    const double k1 = rhs<KIND>(x);
    const double k2 = rhs<KIND>(x + h * (A21 * k1));
    const double k3 = rhs<KIND>(x + h * (A31 * k1 + A32 * k2));
    const double k4 = rhs<KIND>(x + h * (A41 * k1 + A42 * k2 + A43 * k3));
    const double k5 = rhs<KIND>(x + h * (A51 * k1 + A52 * k2 + A53 * k3 + A54 * k4));
    const double k6 = rhs<KIND>(x + h * (A61 * k1 + A62 * k2 + A63 * k3 + A64 * k4 + A65 * k5));
    const double y5 = x + h * (B1 * k1 + B3 * k3 + B4 * k4 + B5 * k5 + B6 * k6);
    const double k7 = rhs<KIND>(y5);
    const double err = h * (E1 * k1 + E3 * k3 + E4 * k4 + E5 * k5 + E6 * k6 + E7 * k7);
    aerr = fabs(err);
    scale = atol + rtol * (fabs(x) + h * fabs(k1));
    return y5;
}

// Running maximum of the ratios a_i / s_i without a division per element:
// the maximum is kept as the pair (num, den) of its element, and a_i / s_i
// exceeds it iff a_i den > num s_i, both products exact up to one rounding
// while every a_i and s_i lies in [2^-500, 2^500) (a_i = 0 included), so the
// element chosen is the one with the largest ratio, up to a tie within an
// ulp.  The thread divides once at the end.  Any value outside that range
// (zero or subnormal scale, NaN, inf, extreme magnitudes) marks the thread,
// which then recomputes its elements' ratios with one division each and the
// NaN-propagating maximum: the result is the plain max_i a_i / s_i either
// way.
struct RatioMax {
    double num = 0.0, den = 1.0;
    bool odd = false;
    __device__ __forceinline__ void add(double a, double sc) {
        // biased exponents (a >= 0: |err|); integer tests, off the FP64 pipe
        const long long ab = __double_as_longlong(a);
        const unsigned ea = (unsigned)(ab >> 52) & 0x7ffu;
        const unsigned es = ((unsigned)__double2hiint(sc) >> 20) & 0x7ffu;
        odd |= !(ab == 0 || ea - 523u < 1000u) || !(es - 523u < 1000u);
        if (a * den > num * sc) {
            num = a;
            den = sc;
        }
    }
};

template <int KIND>
__device__ __forceinline__ double rk4_step(double x, double h) {
    const double k1 = rhs<KIND>(x);
    const double k2 = rhs<KIND>(x + h * (0.5 * k1));
    const double k3 = rhs<KIND>(x + h * (0.5 * k2));
    const double k4 = rhs<KIND>(x + h * k3);
    return x + h * (k1 / 6.0 + k2 / 3.0 + k3 / 3.0 + k4 / 6.0);
}

template <int KIND>
__global__ void __launch_bounds__(256) ode_dp5_attempt_kernel(long long n, double* xa, double* xb, DevCtrl* c,
                                                              unsigned long long cond, int use_cond) {
    __shared__ double red[32];
    __shared__ int s_last;
    const int parity = c->parity;
    const double h = c->dt_try, atol = c->atol, rtol = c->rtol;
    const double* __restrict__ x = parity ? xb : xa;
    double* __restrict__ y = parity ? xa : xb;
    double emax = 0.0;
    if (!c->done) {
        RatioMax m;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            double a, sc;
            y[i] = dp5_attempt<KIND>(x[i], h, atol, rtol, a, sc);
            m.add(a, sc);
        }
        emax = m.num / m.den;
        if (m.odd) {  // exceptional values: the plain maximum of the ratios
            emax = 0.0;
            for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
                 i += (long long)gridDim.x * blockDim.x) {
                double a, sc;
                dp5_attempt<KIND>(x[i], h, atol, rtol, a, sc);
                emax = nanmax(emax, a / sc);
            }
        }
    }
    const double bmax = block_nanmax(emax, red);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(&c->err_bits, bmax);
        __threadfence();
        const unsigned prev = atomicAdd(&c->arrive, 1u);
        s_last = (prev == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const double E = __longlong_as_double((long long)atomicOr(&c->err_bits, 0ull));
        c->err_bits = 0ull;
        c->arrive = 0u;
        int cont = 0;
        if (!c->done) cont = controller_update(c, E);
        if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, cont ? 1u : 0u);
    }
}

template <typename T>
__global__ void copy_if_odd_kernel(const DevCtrl* c, const T* __restrict__ a, T* __restrict__ b, long long n) {
    if (c->parity == 0) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// Adams-Bashforth 4 with RK4 start-up, all steps in registers.
template <int KIND>
__global__ void __launch_bounds__(256) ode_ab4_kernel(long long n, double* x, double dt, long long nsteps) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double u = x[i];
        // history h_j of the last four steps: f_{m-j} itself, or for dx/dt =
        // -x the state x_{m-j} with the sign folded into the update (x' = x -
        // dt sum c_j x_j: the same values as x + dt sum c_j f_j, negation
        // being exact, without an instruction to form -x)
        constexpr bool NEG = KIND == ODE_EXP_DECAY;
        auto hist = [](double v) { return NEG ? v : rhs<KIND>(v); };
        double h0 = 0, h1 = 0, h2 = 0, h3 = 0;
        const long long ns = nsteps < 3 ? nsteps : 3;
        for (long long m = 0; m < ns; ++m) {
            h3 = h2;
            h2 = h1;
            h1 = h0;
            h0 = hist(u);
            u = rk4_step<KIND>(u, dt);
        }
        const double c0 = 55.0 / 24.0, c1 = -59.0 / 24.0, c2 = 37.0 / 24.0, c3 = -9.0 / 24.0;
        for (long long m = ns; m < nsteps; ++m) {
            h3 = h2;
            h2 = h1;
            h1 = h0;
            h0 = hist(u);
            const double sum = c0 * h0 + c1 * h1 + c2 * h2 + c3 * h3;
            u = NEG ? u - dt * sum : u + dt * sum;
        }
        x[i] = u;
    }
}

template <int KIND, int METHOD>
__global__ void __launch_bounds__(256) ode_const_kernel(long long n, double* x, double dt, long long nsteps) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double u = x[i];
        for (long long m = 0; m < nsteps; ++m) {
            if (METHOD == GS_EULER) {
                u = u + dt * rhs<KIND>(u);
            } else if (METHOD == GS_RK4) {
                u = rk4_step<KIND>(u, dt);
            } else {
                double a, sc;  // the error estimate is unused in fixed steps
                u = dp5_attempt<KIND>(u, dt, 1.0, 1.0, a, sc);
            }
        }
        x[i] = u;
    }
}

int sm_count() {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return nsm;
}

template <typename K>
int persistent_grid(K kern, int block, long long n) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, 0);
    if (occ < 1) occ = 1;
    const long long need = (n + block - 1) / block;
    const long long g = std::min<long long>(need, (long long)sm_count() * occ);
    return (int)std::max<long long>(g, 1);
}

#define GCK(call)                              \
    do {                                       \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess) {               \
            set_global_error(e_, #call);       \
            return GS_ERR_CUDA;                \
        }                                      \
    } while (0)

// Workspace layout: [DevCtrl (256 B)] [x' : n doubles, 256-aligned]
constexpr size_t kCtrlBytes = 256;
static_assert(sizeof(DevCtrl) <= kCtrlBytes, "control block must fit its workspace slot");

}  // namespace

extern "C" {

size_t ode_workspace_size(long n) {
    if (n < 0) return 0;
    return kCtrlBytes + ((size_t)n * sizeof(double) + 255) / 256 * 256;
}

gs_status ode_integrate_adaptive(ode_rhs kind, long n, double* x, double* t, double t_end, double* dt,
                                 double atol, double rtol, long max_steps, long* n_acc, long* n_rej,
                                 void* workspace, size_t workspace_bytes, double* dt_log, long log_cap,
                                 void* stream) {
    if ((kind != ODE_EXP_DECAY && kind != ODE_LOGISTIC) || n < 0 || !t || !dt) return GS_ERR_INVALID;
    if (n > 0 && !x) return GS_ERR_INVALID;
    if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < ode_workspace_size(n))
        return GS_ERR_INVALID;
    if (!(atol >= 0) || !(rtol >= 0) || !(atol > 0 || rtol > 0) || !(*dt > 0) || std::isnan(t_end))
        return GS_ERR_INVALID;
    if (log_cap < 0 || (log_cap > 0 && !dt_log)) return GS_ERR_INVALID;
    if (n_acc) *n_acc = 0;
    if (n_rej) *n_rej = 0;
    if (!(*t < t_end) || max_steps == 0 || n == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevCtrl* dc = (DevCtrl*)workspace;
    double* xb = (double*)((unsigned char*)workspace + kCtrlBytes);

    DevCtrl* h = nullptr;
    GCK(cudaMallocHost(&h, sizeof(DevCtrl)));
    memset(h, 0, sizeof(DevCtrl));
    h->mode = CTRL_ADAPTIVE;
    h->t = *t;
    h->t0 = *t;
    h->t_end = t_end;
    h->dt = *dt;
    h->atol = atol;
    h->rtol = rtol;
    h->max_acc = max_steps < 0 ? -1 : max_steps;
    h->max_att = kMaxAttempts;
    h->log_dt = dt_log;
    h->log_cap = log_cap;
    double ht = *dt;
    if (h->t + ht >= t_end) {
        ht = t_end - h->t;
        h->last = 1;
    }
    if (!(ht > 0.0) || h->t + ht == h->t) {
        cudaFreeHost(h);
        return GS_ERR_STEP_UNDERFLOW;
    }
    h->dt_try = ht;

    gs_status st = GS_OK;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMemcpyAsync(dc, h, sizeof(DevCtrl), cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
        cudaGraph_t body = nullptr;
        cudaGraphConditionalHandle hc;
        if ((e = make_while_graph(&g, &hc, &body)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            break;
        if (kind == ODE_EXP_DECAY) {
            auto k = ode_dp5_attempt_kernel<ODE_EXP_DECAY>;
            k<<<persistent_grid(k, 256, n), 256, 0, cap>>>(n, x, xb, dc, (unsigned long long)hc, 1);
        } else {
            auto k = ode_dp5_attempt_kernel<ODE_LOGISTIC>;
            k<<<persistent_grid(k, 256, n), 256, 0, cap>>>(n, x, xb, dc, (unsigned long long)hc, 1);
        }
        cudaError_t el = cudaGetLastError();
        cudaGraph_t tmp = body;
        e = cudaStreamEndCapture(cap, &tmp);
        if (el != cudaSuccess) e = el;
        if (e != cudaSuccess) break;
        if ((e = cudaGraphInstantiate(&ex, g, 0)) != cudaSuccess) break;
        if ((e = cudaGraphLaunch(ex, s)) != cudaSuccess) break;
        copy_if_odd_kernel<double><<<sm_count() * 8, 256, 0, s>>>(dc, xb, x, n);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(h, dc, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    } while (0);
    if (ex) cudaGraphExecDestroy(ex);
    if (g) cudaGraphDestroy(g);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        set_global_error(e, "ode_integrate_adaptive");
        cudaFreeHost(h);
        return GS_ERR_CUDA;
    }
    *t = h->t;
    *dt = h->dt;
    if (n_acc) *n_acc = (long)h->n_acc;
    if (n_rej) *n_rej = (long)h->n_rej;
    st = (gs_status)h->status;
    cudaFreeHost(h);
    return st;
}

gs_status ode_integrate_ab4(ode_rhs kind, long n, double* x, double t0, double dt, long nsteps, void* stream) {
    (void)t0;  // autonomous right-hand sides
    if ((kind != ODE_EXP_DECAY && kind != ODE_LOGISTIC) || n < 0 || nsteps < 0 || !std::isfinite(dt))
        return GS_ERR_INVALID;
    if (n > 0 && !x) return GS_ERR_INVALID;
    if (n == 0 || nsteps == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == ODE_EXP_DECAY) {
        auto k = ode_ab4_kernel<ODE_EXP_DECAY>;
        k<<<persistent_grid(k, 256, n), 256, 0, s>>>(n, x, dt, nsteps);
    } else {
        auto k = ode_ab4_kernel<ODE_LOGISTIC>;
        k<<<persistent_grid(k, 256, n), 256, 0, s>>>(n, x, dt, nsteps);
    }
    GCK(cudaGetLastError());
    return GS_OK;
}

gs_status ode_integrate_const(ode_rhs kind, gs_method method, long n, double* x, double t0, double dt,
                              long nsteps, void* stream) {
    if ((kind != ODE_EXP_DECAY && kind != ODE_LOGISTIC) || n < 0 || nsteps < 0 || !std::isfinite(dt))
        return GS_ERR_INVALID;
    if (method == GS_AB4) return ode_integrate_ab4(kind, n, x, t0, dt, nsteps, stream);
    if (method != GS_EULER && method != GS_RK4 && method != GS_DOPRI5) return GS_ERR_INVALID;
    if (n > 0 && !x) return GS_ERR_INVALID;
    if (n == 0 || nsteps == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
#define ODE_CONST_LAUNCH(K, M)                                               \
    if (kind == K && method == M) {                                          \
        auto k = ode_const_kernel<K, M>;                                     \
        k<<<persistent_grid(k, 256, n), 256, 0, s>>>(n, x, dt, nsteps);      \
    }
    ODE_CONST_LAUNCH(ODE_EXP_DECAY, GS_EULER)
    ODE_CONST_LAUNCH(ODE_EXP_DECAY, GS_RK4)
    ODE_CONST_LAUNCH(ODE_EXP_DECAY, GS_DOPRI5)
    ODE_CONST_LAUNCH(ODE_LOGISTIC, GS_EULER)
    ODE_CONST_LAUNCH(ODE_LOGISTIC, GS_RK4)
    ODE_CONST_LAUNCH(ODE_LOGISTIC, GS_DOPRI5)
#undef ODE_CONST_LAUNCH
    GCK(cudaGetLastError());
    return GS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of ode_integrate_adaptive.
//
// Some callers cannot allocate GPU memory at the time they integrate: code
// that runs under a host application which owns every device allocation
// through its own pool, real-time loops where cudaMalloc's implicit device
// synchronisation and unbounded latency are not allowed, or plugins that may
// only touch memory they were handed.  For them the scratch of the adaptive
// driver (control block + second state buffer) lives in this file-scope
// device array instead of a caller workspace.  Every GPU that loads the
// library holds the array until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr long kStaticMaxElements = 1L << 20;  // 8 MiB of FP64 state
static __device__ __align__(256) unsigned char g_ode_static_scratch[kCtrlBytes + 8 * kStaticMaxElements];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

// Device address of the static scratch for the current device (looked up
// once per device; the host-side symbol is only a stand-in).
cudaError_t static_scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ode_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

__global__ void ctrl_init_kernel(DevCtrl* c, DevCtrl v) { *c = v; }

}  // namespace

extern "C" gs_status ode_integrate_adaptive_noalloc(ode_rhs kind, long n, double* x, double* t, double t_end,
                                                   double* dt, double atol, double rtol, long max_steps,
                                                   long* n_acc, long* n_rej, void* stream) {
    if ((kind != ODE_EXP_DECAY && kind != ODE_LOGISTIC) || n < 0 || !t || !dt) return GS_ERR_INVALID;
    if (n > kStaticMaxElements) {
        set_global_error(cudaErrorInvalidValue,
                         "ode_integrate_adaptive_noalloc: n exceeds the static scratch capacity of 1048576 elements");
        return GS_ERR_INVALID;
    }
    if (n > 0 && !x) return GS_ERR_INVALID;
    if (!(atol >= 0) || !(rtol >= 0) || !(atol > 0 || rtol > 0) || !(*dt > 0) || std::isnan(t_end))
        return GS_ERR_INVALID;
    if (n_acc) *n_acc = 0;
    if (n_rej) *n_rej = 0;
    if (!(*t < t_end) || max_steps == 0 || n == 0) return GS_OK;

    DevCtrl h;
    memset(&h, 0, sizeof(h));
    h.mode = CTRL_ADAPTIVE;
    h.t = *t;
    h.t0 = *t;
    h.t_end = t_end;
    h.dt = *dt;
    h.atol = atol;
    h.rtol = rtol;
    h.max_acc = max_steps < 0 ? -1 : max_steps;
    h.max_att = kMaxAttempts;
    double ht = *dt;
    if (h.t + ht >= t_end) {
        ht = t_end - h.t;
        h.last = 1;
    }
    if (!(ht > 0.0) || h.t + ht == h.t) return GS_ERR_STEP_UNDERFLOW;
    h.dt_try = ht;

    void* base = nullptr;
    GCK(static_scratch_address(&base));
    DevCtrl* dc = (DevCtrl*)base;
    double* xb = (double*)((unsigned char*)base + kCtrlBytes);
    cudaStream_t s = (cudaStream_t)stream;

    // the array keeps the previous call's contents: the whole control block
    // (counters, error accumulator, arrival counter, parity) is rewritten
    ctrl_init_kernel<<<1, 1, 0, s>>>(dc, h);
    GCK(cudaGetLastError());
    int grid = 0;
    if (kind == ODE_EXP_DECAY)
        grid = persistent_grid(ode_dp5_attempt_kernel<ODE_EXP_DECAY>, 256, n);
    else
        grid = persistent_grid(ode_dp5_attempt_kernel<ODE_LOGISTIC>, 256, n);
    // host-driven loop: batches of attempts, then one look at `done`; the
    // attempt kernel does nothing once the run has ended
    const int kBatch = 16;
    int done = 0;
    while (!done) {
        for (int b = 0; b < kBatch; ++b) {
            if (kind == ODE_EXP_DECAY)
                ode_dp5_attempt_kernel<ODE_EXP_DECAY><<<grid, 256, 0, s>>>(n, x, xb, dc, 0ull, 0);
            else
                ode_dp5_attempt_kernel<ODE_LOGISTIC><<<grid, 256, 0, s>>>(n, x, xb, dc, 0ull, 0);
        }
        GCK(cudaGetLastError());
        GCK(cudaMemcpyAsync(&done, &dc->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        GCK(cudaStreamSynchronize(s));
    }
    copy_if_odd_kernel<double><<<sm_count() * 8, 256, 0, s>>>(dc, xb, x, n);
    GCK(cudaGetLastError());
    GCK(cudaMemcpyAsync(&h, dc, sizeof(DevCtrl), cudaMemcpyDeviceToHost, s));
    GCK(cudaStreamSynchronize(s));
    *t = h.t;
    *dt = h.dt;
    if (n_acc) *n_acc = (long)h.n_acc;
    if (n_rej) *n_rej = (long)h.n_rej;
    return (gs_status)h.status;
}
