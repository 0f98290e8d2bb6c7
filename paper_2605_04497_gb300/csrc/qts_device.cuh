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

// The most dynamic shared memory one block may use on sm_103a (227 KB).
constexpr size_t kSmemMax = 227 * 1024;

// Calls with at most this many samples map lanes to (path, sample) pairs
// instead of one sample per lane (which would leave most lanes idle).
constexpr int kFewRows = 16;

// A wait is declared failed after about kWaitNs of GPU time (the global
// nanosecond timer), or after kWaitLimit polls as a backstop (each try_wait
// may suspend for a hardware-defined interval).
constexpr uint64_t kWaitNs = 1000000000ull;
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

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: true when the phase completed; false once about a second has
// passed (or kWaitLimit polls), so a copy that never lands ends as a status
// code instead of a hung context.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_ns() - t0 > kWaitNs) return false;
    }
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
    if constexpr (HAS_NAN) {
        // categorical element (only in ensembles that have them, which always
        // take this variant): x's category in the merged set; NaN by the
        // merged default direction; other values by kOtherOk
        if (bits & kCat) {
            if (x != x) return (bits & kNanOk) != 0;
            if (x >= 0.f && x < 64.f) {
                const int c = (int)x;
                const uint32_t w = __float_as_uint(c < 32 ? lo : hi);
                return ((w >> (c & 31)) & 1u) != 0;
            }
            return (bits & kOtherOk) != 0;
        }
    }
    bool o = (x >= lo) && (x < hi);
    if (HAS_NAN) o = o || ((x != x) && (bits & kNanOk));
    return o;
}

}  // namespace qts

namespace qts {

// Block-level path streaming.  The block's path range [p0, p1) of one bucket
// (D elements + 1 header record per path) is copied into two shared staging
// buffers of `sub` paths each by bulk copies, double-buffered on two
// mbarriers; visit(first_path_index, count, records) runs on every thread for
// each staged sub-chunk.  Thread 0 does the bounded wait and broadcasts the
// outcome, so the decision to stop is block-uniform.  Returns false (after
// reporting QTS_ERR_TIMEOUT and waiting, bounded, for the copies in flight) if
// a copy did not complete.  Must be called by all threads; `bars` must have
// been initialised by mbar_init(.., 1) and a __syncthreads.
template <typename Rec, int D, typename Visit>
__device__ __forceinline__ bool stream_chunks(const Rec* __restrict__ rec, int64_t p0, int64_t p1, int sub,
                                              Rec* st0, Rec* st1, uint64_t* bars, uint32_t* phase_base,
                                              int* s_flag, int* status, Visit&& visit) {
    const int nsub = (int)((p1 - p0 + sub - 1) / sub);
    // phase_base[k] counts completed phases of barrier k before this call, so
    // this routine can be called repeatedly (persistent kernels) on the same bars
    auto issue = [&](int c) {
        const int64_t q0 = p0 + (int64_t)c * sub;
        const int cnt = (int)imin64(sub, p1 - q0);
        const uint32_t bytes = (uint32_t)cnt * (D + 1) * (uint32_t)sizeof(Rec);
        uint64_t* bar = &bars[c & 1];
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s((c & 1) ? (void*)st1 : (void*)st0, rec + q0 * (D + 1), bytes, bar);
    };
    if (threadIdx.x == 0)
        for (int c = 0; c < 2 && c < nsub; ++c) issue(c);
    int failed_at = -1;
    for (int c = 0; c < nsub; ++c) {
        const uint32_t parity = (phase_base[c & 1] + (uint32_t)(c >> 1)) & 1u;
        if (threadIdx.x == 0) *s_flag = mbar_wait_bounded(&bars[c & 1], parity) ? 1 : 0;
        __syncthreads();
        if (!*s_flag) { failed_at = c; break; }
        (void)mbar_try_wait(&bars[c & 1], parity);  // acquire the bulk-copy writes
        const Rec* buf = (c & 1) ? st1 : st0;
        const int64_t q0 = p0 + (int64_t)c * sub;
        visit(q0, (int)imin64(sub, p1 - q0), buf);
        __syncthreads();
        if (threadIdx.x == 0 && c + 2 < nsub) issue(c + 2);
    }
    if (failed_at >= 0) {
        if (threadIdx.x == 0) {
            report(status, QTS_ERR_TIMEOUT);
            for (int c = failed_at; c < failed_at + 2 && c < nsub; ++c)
                (void)mbar_wait_bounded(&bars[c & 1], (phase_base[c & 1] + (uint32_t)(c >> 1)) & 1u);
        }
        __syncthreads();
        return false;
    }
    // advance the phase counters by the number of copies each barrier completed
    if (threadIdx.x == 0) {
        phase_base[0] += (uint32_t)((nsub + 1) / 2);
        phase_base[1] += (uint32_t)(nsub / 2);
    }
    __syncthreads();
    return true;
}

// Lane = sample: warp w calls body(global_path_index, records) for paths w,
// w + nwarps, ... of each staged sub-chunk (every path, when every_warp).
template <typename Rec, int D, typename Body>
__device__ __forceinline__ bool stream_paths(const Rec* __restrict__ rec, int64_t p0, int64_t p1, int sub,
                                             Rec* st0, Rec* st1, uint64_t* bars, uint32_t* phase_base,
                                             int* s_flag, int* status, Body&& body, bool every_warp = false) {
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    return stream_chunks<Rec, D>(rec, p0, p1, sub, st0, st1, bars, phase_base, s_flag, status,
                                 [&](int64_t q0, int cnt, const Rec* buf) {
                                     const int i0 = every_warp ? 0 : warp, di = every_warp ? 1 : nwarps;
                                     for (int i = i0; i < cnt; i += di) body(q0 + i, buf + i * (D + 1));
                                 });
}

// Lane = (path, sample), for calls with few samples: warp w takes `group`
// consecutive paths of [p0, p1) at a time (paths p0 + w group, then every
// nwarps * group), and the lanes of slot k < group work on its k-th path,
// reading the records straight from global memory (each lane its own path:
// no shared staging).  Every lane calls body(global_path_index, records,
// valid); a lane without a path (slot >= group, or past the end) gets the
// step's first path with valid = false and must not write results.  The trip
// count is the same on every lane of a warp, so body may use __syncwarp.
template <typename Rec, int D, typename Body>
__device__ __forceinline__ void walk_paths_grouped(const Rec* __restrict__ rec, int64_t p0, int64_t p1, int group,
                                                   int slot, Body&& body) {
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int64_t i = p0 + (int64_t)warp * group; i < p1; i += (int64_t)nwarps * group) {
        const int64_t k = i + slot;
        const bool valid = slot < group && k < p1;
        const int64_t use = valid ? k : i;
        body(use, rec + use * (D + 1), valid);
    }
}

// Transposed tile of 32 rows of a row-major matrix: tile[c * kTileLd + s] =
// A[(s0 + s) * ld + c] for c < ncols (0 beyond M), plus `extra` zero rows.
// Returns (block-wide) whether any loaded value is NaN.
__device__ __forceinline__ bool load_tile_t(float* tile, const float* __restrict__ A, int64_t s0,
                                            int64_t M, int ncols, int64_t ld, int extra) {
    int nan_seen = 0;
    for (int idx = threadIdx.x; idx < 32 * ncols; idx += blockDim.x) {
        const int s = idx / ncols, c = idx - s * ncols;
        const float v = (s0 + s < M) ? A[(s0 + s) * ld + c] : 0.f;
        tile[c * kTileLd + s] = v;
        nan_seen |= (v != v);
    }
    for (int idx = threadIdx.x; idx < extra * kTileLd; idx += blockDim.x) tile[ncols * kTileLd + idx] = 0.f;
    return __syncthreads_or(nan_seen) != 0;
}

// ntiles transposed tiles of 32 rows each (tile w holds rows s0 + 32 w ..),
// tile w at tile + w * tile_stride, plus `extra` zero rows per tile.
__device__ __forceinline__ bool load_tiles_t(float* tile, const float* __restrict__ A, int64_t s0, int64_t M,
                                             int ncols, int64_t ld, int extra, int ntiles, int tile_stride) {
    int nan_seen = 0;
    for (int idx = threadIdx.x; idx < 32 * ntiles * ncols; idx += blockDim.x) {
        const int s = idx / ncols, c = idx - s * ncols;
        const float v = (s0 + s < M) ? A[(s0 + s) * ld + c] : 0.f;
        tile[(s >> 5) * tile_stride + c * kTileLd + (s & 31)] = v;
        nan_seen |= (v != v);
    }
    for (int idx = threadIdx.x; idx < ntiles * extra * kTileLd; idx += blockDim.x) {
        const int w = idx / (extra * kTileLd), r = idx - w * extra * kTileLd;
        tile[w * tile_stride + ncols * kTileLd + r] = 0.f;
    }
    return __syncthreads_or(nan_seen) != 0;
}

// ------------------------------------------------------- sibling pairs --
//
// Pair tables (FP32 forward, adjoint, batched pass, pairwise interactions)
// hold sibling leaves A, B of a numerical split as one path with val = 1 whose
// last element e (kPairElem) stands for both: for a sample x it gives
// d = val_k - alpha for the leaf k the sample reaches (x in the element's
// interval, then left of theta), -alpha if neither.  h is the path header
// {1, val_A - alpha, val_B - alpha, bits of theta}.
__device__ __forceinline__ void pair_sides(float x, const Rec32& e, const Rec32& h, bool* oa, bool* ob) {
    bool in, left;
    if (x != x) {
        in = (e.bits & kNanOk) != 0;
        left = (e.bits & kDefLeft) != 0;
    } else {
        in = x >= e.lo && x < e.hi;
        left = x < __uint_as_float(h.bits);
    }
    *oa = in && left;
    *ob = in && !left;
}

__device__ __forceinline__ float pair_d(float x, const Rec32& e, const Rec32& h) {
    bool oa, ob;
    pair_sides(x, e, h, &oa, &ob);
    return oa ? h.lo : (ob ? h.hi : -e.z);
}

}  // namespace qts
