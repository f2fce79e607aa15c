// peak.cu -- rogs_measure_fp32_peak: the FP32 fused multiply-add rate of the
// current device, measured (the roofline denominator of the ALU-bound
// compositing kernels; no vendor figure is used).
//
// Every thread runs kChains independent multiply-add recurrences
// a <- a * b + c for `iters` rounds, so that each scheduler always has ready
// FMAs and the FMA pipes, not latency, set the rate.  The grid holds a whole
// number of blocks per SM on every SM.  The recurrences stay bounded
// (|b| < 1) and their sum is written out, so nothing is optimised away.
// FLOPs = 2 per FMA; time = CUDA events around the launch; best of `reps`.
#include "kernels.h"

namespace rogs {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_k(float* __restrict__ sink, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    sink[blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

}  // namespace rogs

extern "C" rogs_status rogs_measure_fp32_peak(int32_t reps, double* tflops, int32_t* sm_count, rogs_stream stream) {
    using namespace rogs;
    if (!tflops || reps < 1) return ROGS_ERR_INVALID;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_k, kPeakThreads, 0) != cudaSuccess)
        return ROGS_ERR_CUDA;
    if (sm_count) *sm_count = sms;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1) * 4;   // four full waves
    const int iters = 2048;
    cudaStream_t s = (cudaStream_t)stream;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rogs_status st = ROGS_OK;
    if (cudaMalloc((void**)&sink, sizeof(float) * (size_t)blocks * kPeakThreads) != cudaSuccess) return ROGS_ERR_OOM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = ROGS_ERR_CUDA;
    double best_ms = 1e30;
    for (int r = 0; r <= reps && st == ROGS_OK; ++r) {   // the first launch warms up
        cudaEventRecord(e0, s);
        fma_peak_k<<<blocks, kPeakThreads, 0, s>>>(sink, iters, 0.999f, 1e-4f);
        note_launches(1);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = ROGS_ERR_CUDA; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms > 0.0f && ms < best_ms) best_ms = ms;
    }
    if (st == ROGS_OK && cudaGetLastError() != cudaSuccess) st = ROGS_ERR_CUDA;
    if (st == ROGS_OK) {
        const double flops = 2.0 * kChains * 4.0 * iters * (double)blocks * kPeakThreads;
        *tflops = flops / (best_ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}
