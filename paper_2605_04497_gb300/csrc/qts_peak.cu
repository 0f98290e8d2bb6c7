// FP32-pipe throughput probe: the denominator of the ALU-bound kernels'
// roofline, measured on the device.  Every thread runs independent chains of
// fused multiply-adds (packed f32x2 or scalar) with full occupancy, so the
// FMA pipe, not dependency latency, bounds the rate; lane operations (one FMA
// on one FP32 lane counts once) per second are reported.

#include "qts_device.cuh"
#include "qts_internal.h"

namespace qts {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;   // independent accumulators per thread
constexpr int kPeakBlocksPerSm = 8;

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float* sink, int iters, float a, float b) {
    float s = 0.f;
    if constexpr (PACKED) {
        float2 acc[kPeakChains];
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) acc[k] = f2(threadIdx.x * 1e-3f + k, 0.5f * k);
        const float2 A = f2s(a), B = f2s(b);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) acc[k] = fma2(acc[k], A, B);
        }
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) s += acc[k].x + acc[k].y;
    } else {
        float acc[2 * kPeakChains];
#pragma unroll
        for (int k = 0; k < 2 * kPeakChains; ++k) acc[k] = threadIdx.x * 1e-3f + k;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 2 * kPeakChains; ++k) acc[k] = fmaf(acc[k], a, b);
        }
#pragma unroll
        for (int k = 0; k < 2 * kPeakChains; ++k) s += acc[k];
    }
    // a sum no chain reaches; it keeps the loop from being removed
    if (s == -1.f) sink[blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

}  // namespace qts

using namespace qts;

extern "C" qts_status qts_fp32_pipe_peak(int32_t packed, double* lane_ops_per_s, qts_stream_t stream) {
    if (!lane_ops_per_s) return fail(QTS_ERR_ARG, "lane_ops_per_s is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = num_sms() * kPeakBlocksPerSm;
    const int iters = 1 << 17;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaMalloc(&sink, sizeof(float) * (size_t)blocks * kPeakThreads);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    float best = 1e30f;
    // one warm-up launch, then the fastest of three
    for (int rep = 0; rep < 4 && ce == cudaSuccess; ++rep) {
        ce = cudaEventRecord(e0, st);
        if (ce == cudaSuccess) {
            if (packed) fma_peak_kernel<true><<<blocks, kPeakThreads, 0, st>>>(sink, iters, 0.999999f, 1e-7f);
            else fma_peak_kernel<false><<<blocks, kPeakThreads, 0, st>>>(sink, iters, 0.999999f, 1e-7f);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce == cudaSuccess && rep > 0) best = std::min(best, ms);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (ce != cudaSuccess) return cuda_fail(ce, "FP32 peak probe");
    const double lane_ops = (double)blocks * kPeakThreads * iters * (2.0 * kPeakChains);
    *lane_ops_per_s = lane_ops / (best * 1e-3);
    return QTS_OK;
}
