// Peak-rate microbenchmarks that the benchmark divides kernel throughputs by
// (no counterpart in the paper): FP32 and FP64 fused multiply-add chains on
// every SM, timed with CUDA events on the caller's stream.
#include "internal.cuh"

namespace polfmm {

constexpr int kPeakChains = 8;     // independent FMA chains per thread
constexpr int kPeakIters = 4096;   // FMAs per chain
constexpr int kPeakThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(R a, R b, R* __restrict__ sink) {
    R x[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) x[k] = R(threadIdx.x + k) * R(1e-3);
#pragma unroll 16
    for (int i = 0; i < kPeakIters; i++)
#pragma unroll
        for (int k = 0; k < kPeakChains; k++) x[k] = fma(x[k], a, b);
    R s = R(0);
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) s += x[k];
    if (s == R(12345.678)) sink[0] = s;  // keeps the chains alive
}

template <typename R>
static int time_fma(cudaStream_t st, int sms, double* tflops) {
    R* sink = nullptr;
    if (dev_alloc(reinterpret_cast<void**>(&sink), sizeof(R)) != cudaSuccess) return POLFMM_ERR_OUT_OF_MEMORY;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = POLFMM_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = POLFMM_ERR_CUDA;
    // 8 blocks of 256 threads per SM: enough warps to hide the FMA latency
    const int grid = 8 * sms;
    const R a = R(0.999999), b = R(1e-7);
    float best = 0.f;
    for (int rep = 0; rc == POLFMM_OK && rep < 4; rep++) {
        cudaEventRecord(e0, st);
        fma_peak_kernel<R><<<grid, kPeakThreads, 0, st>>>(a, b, sink);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = POLFMM_ERR_CUDA;
            break;
        }
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // the first launch warms up
    }
    if (rc == POLFMM_OK && best > 0.f)
        *tflops = 2.0 * kPeakChains * (double)kPeakIters * kPeakThreads * grid / (best * 1e-3) / 1e12;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaGetLastError();
    return rc;
}

}  // namespace polfmm

extern "C" POLFMM_API int fmm_measure_peak(int what, void* cuda_stream, double* tflops) {
    using namespace polfmm;
    if (!tflops || (what != 0 && what != 1)) return POLFMM_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return POLFMM_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return what == 0 ? time_fma<float>(st, sms, tflops) : time_fma<double>(st, sms, tflops);
}
