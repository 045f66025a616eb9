// Arithmetic-rate probe: the FMA throughput of the FP64 or FP32 pipe, measured
// with CUDA events on independent FMA chains spread over every SM.  The plain
// FP64 solve on this part may be bound by FP64 arithmetic rather than by HBM
// (FP64 runs at a small fraction of the FP32 rate), so its roofline needs this
// denominator beside the copy bandwidth.
#include <algorithm>

#include "mx_internal.cuh"

constexpr int PR_CHAINS = 8;      // independent chains per thread (covers the FMA latency)
constexpr int PR_THREADS = 256;

__device__ __forceinline__ float fma_t(float x, float a, float b) { return fmaf(x, a, b); }
__device__ __forceinline__ double fma_t(double x, double a, double b) { return fma(x, a, b); }

template <typename T>
__global__ void __launch_bounds__(PR_THREADS) fma_probe_kernel(T *out, int iters, T a, T b) {
    const int t = blockIdx.x * PR_THREADS + threadIdx.x;
    T x[PR_CHAINS];
#pragma unroll
    for (int c = 0; c < PR_CHAINS; c++) x[c] = T(t) * T(1e-7) + T(c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < PR_CHAINS; c++) x[c] = fma_t(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < PR_CHAINS; c++) s += x[c];
    out[t] = s;  // keeps the chains live; one store per thread
}

template <typename T>
static mx_status probe(int device, double *tflops) {
    int nsm = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return MX_ERR_CUDA;
    }
    const int blocks = nsm * 8;
    const int iters = sizeof(T) == 8 ? 2048 : 16384;
    T *buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mx_status st = MX_OK;
    if (cudaMalloc(&buf, sizeof(T) * blocks * PR_THREADS) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        st = MX_ERR_CUDA;
    }
    double best = 0.0;
    // the multiplier keeps |x| bounded (a fixed point at b / (1 - a)), so no chain overflows
    const T a = T(0.999999), b = T(1e-6);
    for (int rep = 0; st == MX_OK && rep < 4; rep++) {
        cudaEventRecord(e0, 0);
        fma_probe_kernel<T><<<blocks, PR_THREADS>>>(buf, iters, a, b);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = MX_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * PR_CHAINS * double(iters) * blocks * PR_THREADS;
        if (rep > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);  // rep 0 warms up
    }
    if (cudaGetLastError() != cudaSuccess) st = MX_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (st == MX_OK) *tflops = best;
    return st;
}

extern "C" mx_status mx_probe_fma_peak(int device, int fp64, double *tflops) {
    if (!tflops) return MX_ERR_ARG;
    return fp64 ? probe<double>(device, tflops) : probe<float>(device, tflops);
}
