// Device helpers shared by the kernels: packed FP32x2 arithmetic, bulk (TMA)
// copies into shared memory completed on an mbarrier, bounded waits, and the
// shared-memory tile layout.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qts_internal.h"

namespace qts {

// Shared tiles are [row][33] floats: lane (sample) is the column, so a warp
// reading row f touches 32 distinct banks, and the +1 pad makes the transposed
// walk (fixed sample, consecutive rows) conflict-free as well.
constexpr int kTileLd = 33;

// Upper bound on mbarrier polls before a wait is declared failed (each
// try_wait already suspends for a hardware-defined interval).
constexpr uint32_t kWaitLimit = 1u << 24;

// ------------------------------------------------------------ f32x2 ------
// Blackwell executes two FP32 lanes per packed instruction; pairs of
// quadrature nodes share one register pair.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// ------------------------------------------------------------ mbarrier ---
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed; false after kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 1-D bulk copy global -> shared, completion counted on `bar` (the TMA unit
// does the transfer; addresses 16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ void report(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Warp-uniform element bits -> feature index.
__device__ __forceinline__ int feat_of(uint32_t bits) { return (int)(bits & kFeatMask); }

// o_j for one sample: x inside [lo, hi), or x missing and the element's splits
// all send missing values the way the path goes.
template <bool HAS_NAN>
__device__ __forceinline__ bool satisfies(float x, float lo, float hi, uint32_t bits) {
    bool o = (x >= lo) && (x < hi);
    if (HAS_NAN) o = o || ((x != x) && (bits & kNanOk));
    return o;
}

}  // namespace qts
