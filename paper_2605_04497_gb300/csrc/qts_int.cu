// Pairwise Shapley interaction values (Thm 1 with S = {i, j}; Alg. 1 with
// s = 2), in the pred_interactions layout.
//
// For a path with merged elements sorted by feature and a sample,
//     SII_ij += val d_i d_j sum_m w_m prod_{k != i,j} a_k(t_m),   d = o - z,
// computed without division: for each i the running product
// R = P_i * prod_{i<k<j} a_k (P_i = w_m val prod_{k<i} a_k) is extended one
// element at a time and multiplied by the stored suffix S_j = prod_{k>j} a_k.
// This is not a dense contraction (per path a rank-n_quad sum scattered over
// F^2/2 pair slots at density d/F), so it runs on the FP32 pipes, two nodes per
// f32x2 register pair.  Per block (32 samples x a chunk of paths) pair sums
// and first-order sums are accumulated in shared FP32 tiles and flushed into
// FP64 accumulators in the workspace laid out [pair][sample] and
// [feature][sample]; a finalize kernel writes the (F+1) x (F+1) matrices.
//
// qts-build-parts: 6 (part 0: host code; parts 1-5: the per-width kernels)
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "qts_device.cuh"

namespace qts {

// Upper-triangle index of the pair (a, b), a < b < F.
__host__ __device__ __forceinline__ int64_t tri_index(int a, int b, int F) {
    return (int64_t)a * F - (int64_t)a * (a + 1) / 2 + (b - a - 1);
}

struct IntArgs {
    const Rec32* rec;
    int64_t n_paths;
    int64_t paths_per_block;
    int sub;
    int n_tiles;
    const float* X;
    int64_t M;
    int F;
    int cat;            // ensemble has categorical elements: always the NaN-aware variant
    int64_t n_pairs;
    int group;          // few samples (M <= 16): lanes are (path, sample) pairs, a warp
                        // takes `group` = 32 / M paths at a time; 0 otherwise
    double* acc_pair;   // [n_pairs][M]
    double* acc_phi;    // [F][M]
    int* status;
    QuadF q;
};

// the widest register pass a width takes (nodes per pass)
__host__ __device__ constexpr int int_max_np(int D) { return D <= 6 ? 8 : (D <= 12 ? 4 : 2); }

template <int D>
cudaError_t launch_int_d(const IntArgs& a, int np, bool pair_smem, int warps, int64_t blocks, size_t smem,
                         cudaStream_t st);

#if QTS_DEVICE_PARTS

// PAIR_SMEM: pair sums go to a shared tile [n_pairs][33]; otherwise straight to
// the FP64 accumulator (lanes = consecutive samples, so each add is coalesced).
template <int D, int NP, bool HAS_NAN, bool PAIR_SMEM>
__device__ __forceinline__ void int_path_f32(const Rec32* __restrict__ r, const float* __restrict__ xs,
                                             float* ps, float* pt, double* acc_pair, int64_t s,
                                             int64_t M, int lane, int F, const QuadF& q) {
    constexpr int K = NP / 2;
    const float val = r[0].z;
    // a sibling pair (pair tables only): its element sits last, after the
    // padding and out of feature order, with d = val_k - alpha per sample and
    // val = 1 (the pair polynomial is one more linear factor of every term)
    const bool pair = (r[D].bits & kPairElem) != 0;
    float dd[D], c1[D];
    int nreal = D;  // sorted elements before the padding (padding sorts last)
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Rec32 e = r[1 + j];
        const int f = feat_of(e.bits);
        const float x = xs[f * kTileLd + lane];
        const bool o = satisfies<HAS_NAN>(x, e.lo, e.hi, e.bits);
        dd[j] = (o ? 1.f : 0.f) - e.z;
        if (j == D - 1 && pair) dd[j] = pair_d(x, e, r[0]);
        c1[j] = 0.f;
        if (f >= F && j < nreal) nreal = j;
    }
    if (pair && nreal > D - 1) nreal = D - 1;
    const int npass = q.n_pad / NP;
    for (int pass = 0; pass < npass; ++pass) {
        float2 T[K], A[D][K], P[D][K], S[D][K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int m = pass * NP + 2 * k;
            T[k] = f2(q.t[m], q.t[m + 1]);
            P[0][k] = f2(q.w[m] * val, q.w[m + 1] * val);
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float2 z2 = f2s(r[1 + j].z), d2 = f2s(dd[j]);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                A[j][k] = fma2(T[k], d2, z2);
                if (j + 1 < D) P[j + 1][k] = mul2(P[j][k], A[j][k]);
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) S[D - 1][k] = f2s(1.f);
#pragma unroll
        for (int j = D - 1; j >= 1; --j)
#pragma unroll
            for (int k = 0; k < K; ++k) S[j - 1][k] = mul2(S[j][k], A[j][k]);
        // first order: c1_j += sum_m P_j S_j
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float2 a1 = mul2(P[j][0], S[j][0]);
#pragma unroll
            for (int k = 1; k < K; ++k) a1 = fma2(P[j][k], S[j][k], a1);
            c1[j] += a1.x + a1.y;
        }
        // pairs i < j among the sorted elements, then (i, pair element)
#pragma unroll
        for (int i = 0; i < D - 1; ++i) {
            if (i + (pair ? 0 : 1) >= nreal) break;
            const int fi = feat_of(r[1 + i].bits);
            const int64_t rowbase = tri_index(fi, fi + 1, F) - (fi + 1);  // + fj gives the index
            float2 R[K];
#pragma unroll
            for (int k = 0; k < K; ++k) R[k] = P[i][k];
#pragma unroll
            for (int j = i + 1; j < D; ++j) {
                if (j >= nreal) break;
                float2 acc = mul2(R[0], S[j][0]);
#pragma unroll
                for (int k = 1; k < K; ++k) acc = fma2(R[k], S[j][k], acc);
                if (j + 1 < D) {
#pragma unroll
                    for (int k = 0; k < K; ++k) R[k] = mul2(R[k], A[j][k]);
                }
                const float v = (acc.x + acc.y) * (dd[i] * dd[j]);
                const int64_t idx = rowbase + feat_of(r[1 + j].bits);
                if constexpr (PAIR_SMEM) {
                    atomicAdd(&pt[idx * kTileLd + lane], v);
                } else {
                    if (s < M && v != 0.f) atomicAdd(&acc_pair[idx * M + s], (double)v);
                }
            }
            if (pair) {
                // R spans the elements between i and the pair element (padding
                // factors are 1), and the pair element's suffix is 1
                float2 acc = R[0];
#pragma unroll
                for (int k = 1; k < K; ++k) acc = add2(R[k], acc);
                const float v = (acc.x + acc.y) * (dd[i] * dd[D - 1]);
                const int fp = feat_of(r[D].bits);
                const int64_t idx = fi < fp ? tri_index(fi, fp, F) : tri_index(fp, fi, F);
                if constexpr (PAIR_SMEM) {
                    atomicAdd(&pt[idx * kTileLd + lane], v);
                } else {
                    if (s < M && v != 0.f) atomicAdd(&acc_pair[idx * M + s], (double)v);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < D; ++j)
        if (j < nreal || (pair && j == D - 1))
            atomicAdd(&ps[feat_of(r[1 + j].bits) * kTileLd + lane], dd[j] * c1[j]);
}

template <int D, int NP, bool PAIR_SMEM>
__global__ void __launch_bounds__(256) int_kernel(IntArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int F = a.F;
    const size_t rows = F + 1;
    float* xs = (float*)smem;
    float* ps = xs + rows * kTileLd;
    float* pt = ps + rows * kTileLd;
    size_t off = 2 * rows * kTileLd * 4;
    if (PAIR_SMEM) off += (size_t)a.n_pairs * kTileLd * 4;
    off = (off + 15) & ~(size_t)15;
    Rec32* st0 = (Rec32*)(smem + off);
    Rec32* st1 = st0 + (size_t)a.sub * (D + 1);
    uint64_t* bars = (uint64_t*)(st1 + (size_t)a.sub * (D + 1));
    __shared__ int s_flag;
    __shared__ uint32_t s_phase[2];

    const int lane = threadIdx.x & 31;
    const int tile = (int)(blockIdx.x % (unsigned)a.n_tiles);
    const int64_t chunk = blockIdx.x / (unsigned)a.n_tiles;
    const int64_t s0 = (int64_t)tile * 32;
    const int64_t p0 = chunk * a.paths_per_block;
    const int64_t p1 = imin64(p0 + a.paths_per_block, a.n_paths);

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
        s_phase[0] = s_phase[1] = 0;
    }
    for (int idx = threadIdx.x; idx < (int)rows * kTileLd; idx += blockDim.x) ps[idx] = 0.f;
    if (PAIR_SMEM)
        for (int64_t idx = threadIdx.x; idx < a.n_pairs * kTileLd; idx += blockDim.x) pt[idx] = 0.f;
    const bool has_nan = load_tile_t(xs, a.X, s0, a.M, F, F, 1) || a.cat != 0;
    const int64_t s = s0 + lane;

    bool ok;
    if (a.group > 0) {
        // few samples: lane (slot, sample) evaluates path slot of each group for
        // its sample (tile column); the pair and phi tiles take atomics anyway
        const int slot = lane / (int)a.M, col = lane - slot * (int)a.M;
        walk_paths_grouped<Rec32, D>(a.rec, p0, p1, a.group, slot, [&](int64_t, const Rec32* r, bool valid) {
            if (!valid) return;
            if (has_nan) int_path_f32<D, NP, true, PAIR_SMEM>(r, xs, ps, pt, a.acc_pair, col, a.M, col, F, a.q);
            else int_path_f32<D, NP, false, PAIR_SMEM>(r, xs, ps, pt, a.acc_pair, col, a.M, col, F, a.q);
        });
        ok = true;
        __syncthreads();  // every warp's adds are in the tiles before the flush
    } else {
        ok = stream_paths<Rec32, D>(
            a.rec, p0, p1, a.sub, st0, st1, bars, s_phase, &s_flag, a.status,
            [&](int64_t, const Rec32* r) {
                if (has_nan) int_path_f32<D, NP, true, PAIR_SMEM>(r, xs, ps, pt, a.acc_pair, s, a.M, lane, F, a.q);
                else int_path_f32<D, NP, false, PAIR_SMEM>(r, xs, ps, pt, a.acc_pair, s, a.M, lane, F, a.q);
            });
    }
    if (!ok) return;
    // flush: consecutive threads take consecutive samples of one row, so the
    // FP64 adds into the [row][sample] accumulators are coalesced
    for (int idx = threadIdx.x; idx < 32 * F; idx += blockDim.x) {
        const int f = idx >> 5, sl = idx & 31;
        const float v = ps[f * kTileLd + sl];
        if (s0 + sl < a.M && v != 0.f) atomicAdd(&a.acc_phi[(int64_t)f * a.M + s0 + sl], (double)v);
    }
    if (PAIR_SMEM) {
        for (int64_t idx = threadIdx.x; idx < 32 * a.n_pairs; idx += blockDim.x) {
            const int64_t pr = idx >> 5;
            const int sl = (int)(idx & 31);
            const float v = pt[pr * kTileLd + sl];
            if (s0 + sl < a.M && v != 0.f) atomicAdd(&a.acc_pair[pr * a.M + s0 + sl], (double)v);
        }
    }
}

template <int D, int NP, bool PS>
static cudaError_t launch_int_t(const IntArgs& a, int warps, int64_t blocks, size_t smem, cudaStream_t st) {
    auto k = int_kernel<D, NP, PS>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)blocks, warps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// np: nodes per register pass, int_max_np(D), or 4 for widths up to 6 (a
// rule of four points)
template <int D>
cudaError_t launch_int_d(const IntArgs& a, int np, bool pair_smem, int warps, int64_t blocks, size_t smem,
                         cudaStream_t st) {
    constexpr int NP = int_max_np(D);
    if constexpr (NP == 8) {
        if (np < NP) {
            if (pair_smem) return launch_int_t<D, NP / 2, true>(a, warps, blocks, smem, st);
            return launch_int_t<D, NP / 2, false>(a, warps, blocks, smem, st);
        }
    }
    if (pair_smem) return launch_int_t<D, NP, true>(a, warps, blocks, smem, st);
    return launch_int_t<D, NP, false>(a, warps, blocks, smem, st);
}

#define QTS_INST(DD) \
    template cudaError_t launch_int_d<DD>(const IntArgs&, int, bool, int, int64_t, size_t, cudaStream_t);
#if QTS_IN_PART(1)
QTS_INST(32)
#endif
#if QTS_IN_PART(2)
QTS_INST(28)
#endif
#if QTS_IN_PART(3)
QTS_INST(24) QTS_INST(1) QTS_INST(2) QTS_INST(3) QTS_INST(4) QTS_INST(5) QTS_INST(6) QTS_INST(7) QTS_INST(8)
#endif
#if QTS_IN_PART(4)
QTS_INST(20) QTS_INST(9) QTS_INST(10) QTS_INST(11) QTS_INST(12)
#endif
#if QTS_IN_PART(5)
QTS_INST(13) QTS_INST(14) QTS_INST(15) QTS_INST(16)
#endif
#undef QTS_INST

#endif  // QTS_DEVICE_PARTS

#if !QTS_HOST_PART
}  // namespace qts
#endif

#if QTS_HOST_PART

size_t int_smem_bytes(int F, int sub, int D, bool pair_smem) {
    const size_t rows = F + 1;
    size_t off = 2 * rows * kTileLd * 4;
    if (pair_smem) off += (size_t)F * (F - 1) / 2 * kTileLd * 4;
    off = (off + 15) & ~(size_t)15;
    off += 2 * (size_t)sub * (D + 1) * sizeof(Rec32);
    off = (off + 15) & ~(size_t)15;
    return off + 16;
}

// out[s][i][j] (F+1 x F+1, fp32) from the FP64 accumulators; one thread per (s, i).
__global__ void int_finalize_kernel(const double* __restrict__ acc_pair, const double* __restrict__ acc_phi,
                                    int64_t M, int F, double bias, float* __restrict__ out) {
    const int64_t n = M * (F + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t % M;
        const int i = (int)(t / M);
        float* row = out + (s * (F + 1) + i) * (F + 1);
        if (i == F) {
            for (int j = 0; j < F; ++j) row[j] = 0.f;
            row[F] = (float)bias;
            continue;
        }
        double rowsum = 0.0;
        for (int j = 0; j < F; ++j) {
            if (j == i) continue;
            const int a = i < j ? i : j, b = i < j ? j : i;
            const double h = 0.5 * acc_pair[tri_index(a, b, F) * M + s];
            row[j] = (float)h;
            rowsum += h;
        }
        row[i] = (float)(acc_phi[(int64_t)i * M + s] - rowsum);
        row[F] = 0.f;
    }
}

static constexpr size_t kSmemBudget = 200 * 1024;

cudaError_t launch_int_bucket(const qts_ensemble* e, const Bucket& b, bool pairs, const float* X, int64_t M,
                              int F, const QuadF& q, double* acc_pair, double* acc_phi, cudaStream_t st) {
    if (M <= 0 || b.n_paths == 0) return cudaSuccess;
    IntArgs a;
    // pairs: the sibling-pair tables (the bucket is one of e->bprep's)
    a.rec = (pairs ? (const Rec32*)e->bdev.rec : (const Rec32*)e->d_rec) + b.rec_off;
    a.n_paths = b.n_paths;
    a.sub = b.D <= 16 ? 16 : 8;
    // wide inputs: stage fewer paths at a time until the block fits shared memory
    while (a.sub > 1 && int_smem_bytes(F, a.sub, b.D, false) > kSmemMax) a.sub /= 2;
    a.group = M <= kFewRows ? (int)(32 / M) : 0;
    a.paths_per_block = std::max<int64_t>(a.sub, 512 / a.sub * a.sub);
    if (a.group) a.paths_per_block = std::max<int64_t>(a.paths_per_block, 4LL * 4 * a.group);
    a.n_tiles = (int)((M + 31) / 32);
    a.X = X;
    a.M = M;
    a.F = F;
    a.cat = (pairs ? e->bprep.has_cat : e->prep.has_cat) ? 1 : 0;
    a.n_pairs = (int64_t)F * (F - 1) / 2;
    a.acc_pair = acc_pair;
    a.acc_phi = acc_phi;
    a.status = e->d_status;
    a.q = q;
    bool pair_smem = int_smem_bytes(F, a.sub, b.D, true) <= kSmemBudget;
    const size_t smem = int_smem_bytes(F, a.sub, b.D, pair_smem);
    if (smem > kSmemMax) return cudaErrorInvalidConfiguration;
    const int64_t chunks = (b.n_paths + a.paths_per_block - 1) / a.paths_per_block;
    const int64_t blocks = chunks * a.n_tiles;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int warps = 4;
    // nodes per register pass: the width's widest, or half of it when that
    // does not divide the rule's padded node count
    const int np = q.n_pad % int_max_np(b.D) == 0 ? int_max_np(b.D) : int_max_np(b.D) / 2;
    if (q.n_pad % np != 0) return cudaErrorInvalidValue;
    switch (b.D) {
#define QTS_CASE(DD) \
    case DD: return launch_int_d<DD>(a, np, pair_smem, warps, blocks, smem, st);
        QTS_CASE(1) QTS_CASE(2) QTS_CASE(3) QTS_CASE(4) QTS_CASE(5) QTS_CASE(6) QTS_CASE(7)
        QTS_CASE(8) QTS_CASE(9) QTS_CASE(10) QTS_CASE(11) QTS_CASE(12) QTS_CASE(13) QTS_CASE(14)
        QTS_CASE(15) QTS_CASE(16) QTS_CASE(20) QTS_CASE(24) QTS_CASE(28) QTS_CASE(32)
#undef QTS_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_int_finalize(const double* acc_pair, const double* acc_phi, int64_t M, int F,
                                double bias, float* out, cudaStream_t st) {
    const int64_t n = M * (F + 1);
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8 * 152);
    int_finalize_kernel<<<blocks, 256, 0, st>>>(acc_pair, acc_phi, M, F, bias, out);
    return cudaGetLastError();
}

}  // namespace qts

using namespace qts;

extern "C" qts_status qts_shap_interactions(qts_ensemble* e, const float* X, int64_t M, int32_t F,
                                            int32_t n_quad, float* phi_ij, qts_stream_t stream) {
    qts_status st = check_call(e, X, M, F, n_quad);
    if (st != QTS_OK) return st;
    if (M == 0) return QTS_OK;
    if (!phi_ij) return fail(QTS_ERR_ARG, "phi_ij is NULL");
    if (e->flags & QTS_FLAG_FP64)
        return fail(QTS_ERR_UNSUPPORTED, "interactions are computed with the FP32 tables only");
    if (e->prep.max_unique > 32)
        return fail(QTS_ERR_UNSUPPORTED, "interactions support paths of at most 32 unique features");
    cudaStream_t s = (cudaStream_t)stream;
    if (n_quad != QTS_NQ_EXACT && (n_quad < 1 || n_quad > QTS_MAX_QUAD)) return fail(QTS_ERR_ARG, "quadrature rule");
    // the sibling-pair tables (built on the first call that needs them)
    st = ensure_batch_tables(e);
    if (st != QTS_OK) return st;
    const int64_t n_pairs = (int64_t)F * (F - 1) / 2;
    const size_t bytes = sizeof(double) * (size_t)((n_pairs + F) * M);
    st = ensure_workspace(e, bytes);
    if (st != QTS_OK) return st;
    double* acc_pair = (double*)e->d_work;
    double* acc_phi = acc_pair + n_pairs * M;
    cudaError_t ce = cudaMemsetAsync(e->d_work, 0, bytes, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "workspace clear");
    for (const Bucket& b : e->bprep.buckets) {
        // the bucket's rule, padded to 4 nodes up to width 12 (a pass of 4 or 8
        // nodes) and to 2 above.  QTS_NQ_EXACT: the pair terms need
        // ceil((D - 1) / 2) points, but the diagonal holds first-order values,
        // so the kernel takes the first-order count ceil(D / 2) (Thm 2)
        QuadF qf;
        if (!make_quad(nodes_for(n_quad, b.D, 1), &qf, nullptr, b.D <= 12 ? 4 : 2))
            return fail(QTS_ERR_ARG, "quadrature rule");
        ce = launch_int_bucket(e, b, true, X, M, F, qf, acc_pair, acc_phi, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "interaction kernel launch");
    }
    ce = launch_int_finalize(acc_pair, acc_phi, M, F, e->bprep.bias, phi_ij, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "interaction finalize launch");
    return QTS_OK;
}

// ------------------------------------------------- allocation-free variant --
//
// Same kernels as qts_shap_interactions, but the FP64 accumulators live in a
// fixed device array that is part of the library image, so the call never
// allocates.  Host code cannot use the array's name as a device pointer: its
// address comes from cudaGetSymbolAddress, with the device current.  That
// address belongs to a context - a device reset destroys the primary context,
// the next call creates a new one, reloads the library's module, and the array
// may then sit elsewhere - so the looked-up address is cached under the current
// context's process-unique id (cuCtxGetId), not under the device ordinal.  The
// two driver calls are fetched through the runtime, so the library still links
// no driver library of its own.

namespace qts {

constexpr int64_t kNoAllocDoubles = (int64_t)2 * 1024 * 1024;  // 16 MiB per device

static __device__ __align__(256) double g_int_noalloc_scratch[kNoAllocDoubles];

struct CtxFns {
    PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    PFN_cuCtxGetId_v12000 get_id = nullptr;
};

static CtxFns ctx_fns() {
    static CtxFns f;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f.get_current = (PFN_cuCtxGetCurrent_v4000)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f.get_id = (PFN_cuCtxGetId_v12000)p;
        cudaGetLastError();  // a missing entry point is not an error of the caller's next call
    });
    return f;
}

// Unique id of the context current on this thread; false when there is none
// (the runtime has not made one current yet) or the driver cannot say.
static bool current_ctx_id(unsigned long long* id) {
    const CtxFns f = ctx_fns();
    if (!f.get_current || !f.get_id) return false;
    CUcontext ctx = nullptr;
    if (f.get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return f.get_id(ctx, id) == CUDA_SUCCESS;
}

static std::mutex g_noalloc_mu;
static std::vector<std::pair<unsigned long long, void*>> g_noalloc_ptr;  // (context id, address)

static qts_status noalloc_scratch(void** out) {
    unsigned long long id = 0;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (current_ctx_id(&id)) {
        for (const auto& kv : g_noalloc_ptr)
            if (kv.first == id) {
                *out = kv.second;
                return QTS_OK;
            }
    }
    void* p = nullptr;
    cudaError_t ce = cudaGetSymbolAddress(&p, g_int_noalloc_scratch);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetSymbolAddress of the interaction scratch");
    // the lookup makes the device's context current if none was: ask again;
    // without an id the address is not cached and is looked up on every call
    if (current_ctx_id(&id)) g_noalloc_ptr.emplace_back(id, p);
    *out = p;
    return QTS_OK;
}

}  // namespace qts

extern "C" qts_status qts_shap_interactions_noalloc(qts_ensemble* e, const float* X, int64_t M, int32_t F,
                                                    int32_t n_quad, float* phi_ij, qts_stream_t stream) {
    qts_status st = check_call(e, X, M, F, n_quad);
    if (st != QTS_OK) return st;
    if (M == 0) return QTS_OK;
    if (!phi_ij) return fail(QTS_ERR_ARG, "phi_ij is NULL");
    if (e->flags & QTS_FLAG_FP64)
        return fail(QTS_ERR_UNSUPPORTED, "interactions are computed with the FP32 tables only");
    if (e->prep.max_unique > 32)
        return fail(QTS_ERR_UNSUPPORTED, "interactions support paths of at most 32 unique features");
    const int64_t n_pairs = (int64_t)F * (F - 1) / 2;
    const int64_t need = (n_pairs + F) * M;
    if (need > kNoAllocDoubles)
        return fail(QTS_ERR_UNSUPPORTED,
                    "qts_shap_interactions_noalloc needs (F(F-1)/2 + F) * M = " + std::to_string(need) +
                        " accumulator doubles; the fixed scratch holds " + std::to_string(kNoAllocDoubles) +
                        " (use qts_shap_interactions for larger calls)");
    cudaStream_t s = (cudaStream_t)stream;
    // QTS_NQ_EXACT: exact for the ensemble's widest path; first-order count,
    // because the diagonal holds first-order values (Thm 2)
    QuadF qf;
    if (!make_quad(nodes_for(n_quad, e->prep.max_unique, 1), &qf, nullptr))
        return fail(QTS_ERR_ARG, "quadrature rule");
    void* scratch = nullptr;
    st = noalloc_scratch(&scratch);
    if (st != QTS_OK) return st;
    double* acc_pair = (double*)scratch;
    double* acc_phi = acc_pair + n_pairs * M;
    // the array keeps the previous call's sums: clear the part this call uses
    cudaError_t ce = cudaMemsetAsync(scratch, 0, sizeof(double) * (size_t)need, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "scratch clear");
    for (const Bucket& b : e->prep.buckets) {
        ce = launch_int_bucket(e, b, false, X, M, F, qf, acc_pair, acc_phi, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "interaction kernel launch");
    }
    ce = launch_int_finalize(acc_pair, acc_phi, M, F, e->prep.bias, phi_ij, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "interaction finalize launch");
    return QTS_OK;
}

#endif  // QTS_HOST_PART
