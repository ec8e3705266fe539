// Measured FP64 and FP32 fused multiply-add issue rates of the current device: the
// denominators of the FP-issue rooflines of the sweep kernels.  The FP64 sweep on this part
// is bound by FP64 instruction issue (every addition of its tree is issued as an FMA), and
// the temporally blocked FP32 sweep by FP32 instruction issue, so their achieved instruction
// rates are reported against what a plain FMA stream reaches on the same device.
//
// Each thread runs kChains independent dependent chains a <- fma(a, x, y) (enough
// independent instructions to cover the pipes' latency), every SM runs kBlocksPerSm blocks
// of 256 threads, and the rate is FMAs issued / CUDA-event time of one launch after a
// warm-up launch.  x and y keep every chain bounded (|a| stays below 2), so no value becomes
// subnormal, infinite or NaN.  The chains' results only reach memory behind a test the
// compiler cannot decide, so the loop is not removed.
#include <cstdio>

#include "cj_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__device__ double g_peak_sink64;
__device__ float g_peak_sink32;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_stream(long long iters, T x, T y, T *sink) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], x, y);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == (T)-12345.0) *sink = s;  // never true; keeps the chains live
}

template <typename T>
cudaError_t time_stream(long long iters, int blocks, T *sink, cudaStream_t s, double *rate) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    const T x = (T)0.5, y = (T)0.25;  // fixed point 0.5: every chain contracts towards it
    fma_stream<T><<<blocks, kThreads, 0, s>>>(iters / 8 + 1, x, y, sink);  // warm-up
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        fma_stream<T><<<blocks, kThreads, 0, s>>>(iters, x, y, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess)
        *rate = (double)blocks * kThreads * kChains * (double)iters / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" cj_status cj_issue_peaks(void *stream, double *fp64_tfma, double *fp32_tfma) {
    if (!fp64_tfma && !fp32_tfma) return CJ_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cj_issue_peaks: device");
        return CJ_ERR_CUDA;
    }
    const int blocks = sms * kBlocksPerSm;
    cudaStream_t s = (cudaStream_t)stream;
    if (fp64_tfma) {
        double *sink = nullptr;
        e = cudaGetSymbolAddress((void **)&sink, g_peak_sink64);
        // ~0.6 T FP64 FMA/s: 3 * 2^13 iterations x 8 chains x 155,648 threads ~ 50 ms
        if (e == cudaSuccess) e = time_stream<double>(3 << 13, blocks, sink, s, fp64_tfma);
        if (e != cudaSuccess) {
            set_cuda_error(e, "cj_issue_peaks: FP64 stream");
            return CJ_ERR_CUDA;
        }
    }
    if (fp32_tfma) {
        float *sink = nullptr;
        e = cudaGetSymbolAddress((void **)&sink, g_peak_sink32);
        // ~37 T FP32 FMA/s: 3 * 2^19 iterations ~ 50 ms
        if (e == cudaSuccess) e = time_stream<float>(3 << 19, blocks, sink, s, fp32_tfma);
        if (e != cudaSuccess) {
            set_cuda_error(e, "cj_issue_peaks: FP32 stream");
            return CJ_ERR_CUDA;
        }
    }
    return CJ_OK;
}
