// algebra.cu -- the n-ary stage algebra (section "The distributed OpenFPM
// state type and algebra": for_each operations over up to 15 states) and the
// context-free utilities of the library (error text, FP64 peak probe).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "gs_internal.h"
#include "host_util.h"

namespace {

thread_local char g_err[512] = {0};

constexpr int kMaxTerms = 15;

template <typename T>
struct AxpyArgs {
    const T* x[kMaxTerms];
    T a[kMaxTerms];
    T* y;
    long long n;
    int nterms;
};

// y = sum_j a_j x_j.  Each thread owns whole 16-byte vectors (one 16-byte
// load per operand, one store), then a scalar tail.  y may alias an operand:
// every element is read before it is written by the same thread.
template <typename T, int NT>
__global__ void __launch_bounds__(256) axpy_kernel(const AxpyArgs<T> A) {
    constexpr int V = 16 / sizeof(T);
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const long long nv = A.n / V;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += stride) {
        T acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = T(0);
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const VT q = reinterpret_cast<const VT*>(A.x[j])[i];
            const T* qs = reinterpret_cast<const T*>(&q);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += A.a[j] * qs[v];
        }
        VT o;
        T* os = reinterpret_cast<T*>(&o);
#pragma unroll
        for (int v = 0; v < V; ++v) os[v] = acc[v];
        reinterpret_cast<VT*>(A.y)[i] = o;
    }
    for (long long i = nv * V + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < A.n; i += stride) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < NT; ++j) acc += A.a[j] * A.x[j][i];
        A.y[i] = acc;
    }
}

template <typename T, int NT>
cudaError_t launch_axpy_nt(const AxpyArgs<T>& A, cudaStream_t s) {
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, axpy_kernel<T, NT>, 256, 0);
    if (occ < 1) occ = 1;
    const long long work = std::max<long long>(A.n / (16 / (long long)sizeof(T)), 1);
    const int grid = (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, (long long)nsm * occ));
    axpy_kernel<T, NT><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpy(const AxpyArgs<T>& A, cudaStream_t s) {
    switch (A.nterms) {
#define AXPY_CASE(K) \
    case K: return launch_axpy_nt<T, K>(A, s);
        AXPY_CASE(1) AXPY_CASE(2) AXPY_CASE(3) AXPY_CASE(4) AXPY_CASE(5)
        AXPY_CASE(6) AXPY_CASE(7) AXPY_CASE(8) AXPY_CASE(9) AXPY_CASE(10)
        AXPY_CASE(11) AXPY_CASE(12) AXPY_CASE(13) AXPY_CASE(14) AXPY_CASE(15)
#undef AXPY_CASE
        default: return cudaErrorInvalidValue;
    }
}

// FP64 FMA throughput: 8 independent dependent-chains per thread.
__global__ void __launch_bounds__(256) fp64_fma_probe(double* out, int iters, double a, double b) {
    double r[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = threadIdx.x * 1e-3 + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) r[j] = fma(r[j], a, b);
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += r[j];
    if (s == 12345.678) out[0] = s;  // keeps the chains live
}

}  // namespace

void set_global_error(cudaError_t e, const char* where) {
    snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
}

extern "C" {

const char* gs_last_global_error(void) { return g_err; }

gs_status ode_axpy_stage(long n, gs_precision prec, int nterms, const double* coef, const void* const* x,
                         void* y, void* stream) {
    if (n < 0 || nterms < 1 || nterms > kMaxTerms || !coef || !x) return GS_ERR_INVALID;
    if (prec != GS_FP32 && prec != GS_FP64) return GS_ERR_INVALID;
    if (n == 0) return GS_OK;
    if (!y || ((uintptr_t)y & 15)) return GS_ERR_INVALID;
    for (int j = 0; j < nterms; ++j)
        if (!x[j] || ((uintptr_t)x[j] & 15)) return GS_ERR_INVALID;
    cudaError_t e;
    if (prec == GS_FP64) {
        AxpyArgs<double> A;
        memset(&A, 0, sizeof(A));
        for (int j = 0; j < nterms; ++j) {
            A.x[j] = (const double*)x[j];
            A.a[j] = coef[j];
        }
        A.y = (double*)y;
        A.n = n;
        A.nterms = nterms;
        e = launch_axpy(A, (cudaStream_t)stream);
    } else {
        AxpyArgs<float> A;
        memset(&A, 0, sizeof(A));
        for (int j = 0; j < nterms; ++j) {
            A.x[j] = (const float*)x[j];
            A.a[j] = (float)coef[j];
        }
        A.y = (float*)y;
        A.n = n;
        A.nterms = nterms;
        e = launch_axpy(A, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) {
        set_global_error(e, "ode_axpy_stage");
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

gs_status gs_measure_fp64_peak(double* tflops, void* stream) {
    if (!tflops) return GS_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    cudaError_t e;
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    const int blocks_per_sm = 8, threads = 256, iters = 4096;
    do {
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) break;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) break;
        if ((e = cudaMalloc(&out, sizeof(double))) != cudaSuccess) break;
        if ((e = cudaEventCreate(&e0)) != cudaSuccess) break;
        if ((e = cudaEventCreate(&e1)) != cudaSuccess) break;
        const int grid = nsm * blocks_per_sm;
        fp64_fma_probe<<<grid, threads, 0, s>>>(out, iters / 4, 1.0000001, 1e-9);  // warm-up
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
        fp64_fma_probe<<<grid, threads, 0, s>>>(out, iters, 1.0000001, 1e-9);
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        const double fmas = (double)grid * threads * iters * 8.0;
        *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    } while (0);
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_global_error(e, "gs_measure_fp64_peak");
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

}  // extern "C"
