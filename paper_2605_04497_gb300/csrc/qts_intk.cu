// Shapley interaction indices of any order s (Thm 1 with |S| = s; Alg. 1 with
// general s; exact for paths of at most 2 n + s - 1 unique features by Thm 2).
//
// For a path with elements sorted by feature and chosen positions
// c_1 < ... < c_s,
//     SII_S += val prod_i d_{c_i} sum_m w_m prod_{l not chosen} a_l(t_m),
// and the excluded product is P_{c_1} * prod_{c_1<l<c_2} a_l * ... * S_{c_s}:
// running products against the stored suffixes S, no division.  The orders
// 4-8 have too many subsets per path to unroll, so each warp keeps its lanes'
// d_l and S_l in shared memory, the subset loops stay rolled, and a template
// recursion over the remaining order gives every level its own running product
// in registers.  Subsets are stored compactly in lexicographic order of their
// sorted features and accumulated in FP64 in the workspace, laid out
// [subset][sample]; a finalize kernel writes [sample][subset] in FP32.
//
// qts-build-parts: 5 (part 0: host code; parts 1-4: the per-width kernels)
#include <algorithm>
#include <string>

#include "qts_device.cuh"

namespace qts {

constexpr int kIntkWarps = 4;
constexpr int kIntkMaxD = 16;
constexpr int kIntkPairs = 4;  // node pairs per pass: all 8 nodes, one atomic per subset

// C(n, R) for a compile-time R; 0 when n < R.
template <int R>
__host__ __device__ __forceinline__ int64_t binom_r(int64_t n) {
    if (n < R) return 0;
    int64_t v = 1;
#pragma unroll
    for (int i = 1; i <= R; ++i) v = v * (n - R + i) / i;
    return v;
}

struct IntkArgs {
    const Rec32* rec;
    int64_t n_paths;
    int64_t paths_per_block;
    int sub;
    int n_tiles;
    const float* X;
    int64_t M;
    int F;
    int cat;            // ensemble has categorical elements: always the NaN-aware variant
    int order;
    int group;          // few samples (M <= 16): lanes are (path, sample) pairs, a warp
                        // takes `group` = 32 / M paths at a time; 0 otherwise
    double* acc;        // [C(F, order)][M]
    int* status;
    QuadF q;
};

// Per-warp view of one path for the subset recursion.
struct IntkPath {
    const Rec32* r;     // the path's records (header, elements) in shared memory
    const float* dd;    // [element][32] d = o - z of the lane's sample
    const float2* S;    // [element][pair][32] suffix products at this pass's nodes
    const int* fe;      // feature of element j at fe[j * fe_ld] (fe_ld 1: warp-uniform;
    int fe_ld;          // 32: this lane's own path, when lanes hold different paths)
    float2 T[kIntkPairs];  // this pass's nodes
    int nreal;          // elements with a real feature (padding excluded)
    int F;
    int lane;
    bool live;
    int64_t s, M;
    double* acc;
};

// Shared-memory layout of a block, every part 16-byte aligned: per-warp S
// (float2) and d (float) slices, per-warp features, the x tile, the two path
// staging buffers and the barriers.
struct IntkSmem {
    size_t S, dd, fe, xs, st, bars, total;
};

__host__ __device__ __forceinline__ size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

__host__ __device__ __forceinline__ IntkSmem intk_smem(int F, int sub, int D) {
    IntkSmem L;
    L.S = 0;
    L.dd = align16(L.S + (size_t)kIntkWarps * kIntkMaxD * kIntkPairs * 32 * sizeof(float2));
    L.fe = align16(L.dd + (size_t)kIntkWarps * kIntkMaxD * 32 * sizeof(float));
    L.xs = align16(L.fe + (size_t)kIntkWarps * kIntkMaxD * 32 * sizeof(int));
    L.st = align16(L.xs + (size_t)(F + 1) * kTileLd * sizeof(float));
    L.bars = align16(L.st + 2 * (size_t)sub * (D + 1) * sizeof(Rec32));
    L.total = L.bars + 2 * sizeof(uint64_t);
    return L;
}

template <int D>
cudaError_t launch_intk_d(const IntkArgs& a, int64_t blocks, size_t smem, cudaStream_t st);

#if QTS_DEVICE_PARTS

// Choose the next element at position >= start with REM more to follow.  R is
// the product of the unchosen elements before `start` (times w val), dp the
// product of the chosen elements' d, rank the lexicographic rank so far.
template <int REM>
__device__ __forceinline__ void intk_choose(const IntkPath& c, int start, const float2 (&R0)[kIntkPairs],
                                            float dp, int64_t rank, int prev) {
    float2 R[kIntkPairs];
#pragma unroll
    for (int k = 0; k < kIntkPairs; ++k) R[k] = R0[k];
#pragma unroll 1
    for (int j = start; j + REM < c.nreal; ++j) {
        const int f = c.fe[j * c.fe_ld];
        const float d = c.dd[j * 32 + c.lane];
        // subsets that agree so far and take a smaller feature here come first
        const int64_t rk = rank + binom_r<REM + 1>(c.F - prev - 1) - binom_r<REM + 1>(c.F - f);
        if constexpr (REM == 0) {
            const float2* Sj = c.S + (size_t)j * kIntkPairs * 32 + c.lane;
            float2 t = mul2(R[0], Sj[0]);
#pragma unroll
            for (int k = 1; k < kIntkPairs; ++k) t = fma2(R[k], Sj[k * 32], t);
            const float v = (t.x + t.y) * dp * d;
            if (c.live && v != 0.f) atomicAdd(&c.acc[rk * c.M + c.s], (double)v);
        } else {
            intk_choose<REM - 1>(c, j + 1, R, dp * d, rk, f);
        }
        const float2 z2 = f2s(c.r[1 + j].z), d2 = f2s(d);
#pragma unroll
        for (int k = 0; k < kIntkPairs; ++k) R[k] = mul2(R[k], fma2(c.T[k], d2, z2));  // j stays unchosen
    }
}

// lane: the lane's slot in the per-warp dd / S / fe arrays; col: its sample's
// column of the x tile; grouped: lanes hold different paths (r is per lane,
// features go to fe[j * 32 + lane]); live = false: compute, do not add.
template <int D, bool HAS_NAN>
__device__ __forceinline__ void intk_path(const Rec32* __restrict__ r, const float* __restrict__ xs, float* dd,
                                          float2* S, int* fe, const IntkArgs& a, int64_t s, int lane, int col,
                                          bool grouped, bool live) {
    const int F = a.F;
    int nreal = D;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Rec32 e = r[1 + j];
        const int f = feat_of(e.bits);
        const bool o = satisfies<HAS_NAN>(xs[f * kTileLd + col], e.lo, e.hi, e.bits);
        dd[j * 32 + lane] = (o ? 1.f : 0.f) - e.z;
        if (grouped) fe[j * 32 + lane] = f;
        else if (lane == 0) fe[j] = f;
        if (f >= F && j < nreal) nreal = j;
    }
    __syncwarp();
    if (nreal >= a.order) {  // widths <= 16 have no padding: the same on every lane
        IntkPath c{r, dd, S, grouped ? fe + lane : fe, grouped ? 32 : 1, {}, nreal, F, lane, live && s < a.M, s,
                   a.M, a.acc};
        const float val = r[0].z;
        for (int m0 = 0; m0 < a.q.n_pad; m0 += 2 * kIntkPairs) {
            float2 R0[kIntkPairs], suf[kIntkPairs];
#pragma unroll
            for (int k = 0; k < kIntkPairs; ++k) {
                c.T[k] = f2(a.q.t[m0 + 2 * k], a.q.t[m0 + 2 * k + 1]);
                R0[k] = f2(a.q.w[m0 + 2 * k] * val, a.q.w[m0 + 2 * k + 1] * val);
                suf[k] = f2s(1.f);
            }
            // suffix products S_j = prod_{l > j} a_l at this pass's nodes
#pragma unroll
            for (int j = D - 1; j >= 0; --j) {
                const float2 z2 = f2s(r[1 + j].z), d2 = f2s(dd[j * 32 + lane]);
#pragma unroll
                for (int k = 0; k < kIntkPairs; ++k) {
                    S[((size_t)j * kIntkPairs + k) * 32 + lane] = suf[k];
                    suf[k] = mul2(suf[k], fma2(c.T[k], d2, z2));
                }
            }
            switch (a.order) {
                case 2: intk_choose<1>(c, 0, R0, 1.f, 0, -1); break;
                case 3: intk_choose<2>(c, 0, R0, 1.f, 0, -1); break;
                case 4: intk_choose<3>(c, 0, R0, 1.f, 0, -1); break;
                case 5: intk_choose<4>(c, 0, R0, 1.f, 0, -1); break;
                case 6: intk_choose<5>(c, 0, R0, 1.f, 0, -1); break;
                case 7: intk_choose<6>(c, 0, R0, 1.f, 0, -1); break;
                case 8: intk_choose<7>(c, 0, R0, 1.f, 0, -1); break;
                default: break;
            }
        }
    }
    __syncwarp();  // dd, S and fe are rewritten by the warp's next path
}

template <int D>
__global__ void __launch_bounds__(kIntkWarps * 32) intk_kernel(IntkArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int F = a.F;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const IntkSmem L = intk_smem(F, a.sub, D);
    float2* S_all = (float2*)(smem + L.S);
    float* dd_all = (float*)(smem + L.dd);
    int* fe_all = (int*)(smem + L.fe);
    float* xs = (float*)(smem + L.xs);
    Rec32* st0 = (Rec32*)(smem + L.st);
    Rec32* st1 = st0 + (size_t)a.sub * (D + 1);
    uint64_t* bars = (uint64_t*)(smem + L.bars);
    __shared__ int s_flag;
    __shared__ uint32_t s_phase[2];
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
    const bool has_nan = load_tile_t(xs, a.X, s0, a.M, F, F, 1) || a.cat != 0;
    const int64_t s = s0 + lane;
    float2* S = S_all + (size_t)warp * kIntkMaxD * kIntkPairs * 32;
    float* dd = dd_all + (size_t)warp * kIntkMaxD * 32;
    int* fe = fe_all + (size_t)warp * kIntkMaxD * 32;
    if (a.group > 0) {
        // few samples: lane (slot, sample) evaluates path slot of each group for
        // its sample; lanes without a path follow along without adding
        const int slot = lane / (int)a.M, col = lane - slot * (int)a.M;
        walk_paths_grouped<Rec32, D>(a.rec, p0, p1, a.group, slot, [&](int64_t, const Rec32* r, bool valid) {
            if (has_nan) intk_path<D, true>(r, xs, dd, S, fe, a, col, lane, col, true, valid);
            else intk_path<D, false>(r, xs, dd, S, fe, a, col, lane, col, true, valid);
        });
        return;
    }
    (void)stream_paths<Rec32, D>(a.rec, p0, p1, a.sub, st0, st1, bars, s_phase, &s_flag, a.status,
                                 [&](int64_t, const Rec32* r) {
                                     if (has_nan) intk_path<D, true>(r, xs, dd, S, fe, a, s, lane, lane, false, true);
                                     else intk_path<D, false>(r, xs, dd, S, fe, a, s, lane, lane, false, true);
                                 });
}

template <int D>
cudaError_t launch_intk_d(const IntkArgs& a, int64_t blocks, size_t smem, cudaStream_t st) {
    auto k = intk_kernel<D>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)blocks, kIntkWarps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

#define QTS_INST(DD) \
    template cudaError_t launch_intk_d<DD>(const IntkArgs&, int64_t, size_t, cudaStream_t);
#if QTS_IN_PART(1)
QTS_INST(2) QTS_INST(3) QTS_INST(4) QTS_INST(5)
#endif
#if QTS_IN_PART(2)
QTS_INST(6) QTS_INST(7) QTS_INST(8) QTS_INST(9)
#endif
#if QTS_IN_PART(3)
QTS_INST(10) QTS_INST(11) QTS_INST(12) QTS_INST(13)
#endif
#if QTS_IN_PART(4)
QTS_INST(14) QTS_INST(15) QTS_INST(16)
#endif
#undef QTS_INST

#endif  // QTS_DEVICE_PARTS

#if !QTS_HOST_PART
}  // namespace qts
#endif

#if QTS_HOST_PART

constexpr int kIntkMaxOrder = 8;

static int64_t binom_host(int64_t n, int k) {
    if (k < 0 || n < k) return 0;
    int64_t v = 1;
    for (int i = 1; i <= k; ++i) v = v * (n - k + i) / i;
    return v;
}

// out[s][t] = acc[t][s] (FP64 -> FP32), one thread per (subset, sample).
__global__ void intk_finalize_kernel(const double* __restrict__ acc, int64_t M, int64_t n_sub,
                                     float* __restrict__ out) {
    const int64_t n = M * n_sub;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / M, s = i - t * M;
        out[s * n_sub + t] = (float)acc[i];
    }
}

static cudaError_t launch_intk_bucket(const qts_ensemble* e, const Bucket& b, const float* X, int64_t M, int F,
                                      int order, const QuadF& q, double* acc, cudaStream_t st) {
    if (M <= 0 || b.n_paths == 0 || b.D < order) return cudaSuccess;
    IntkArgs a;
    a.rec = (const Rec32*)e->d_rec + b.rec_off;
    a.n_paths = b.n_paths;
    a.sub = 16;
    a.paths_per_block = 128;
    a.n_tiles = (int)((M + 31) / 32);
    a.group = M <= kFewRows ? (int)(32 / M) : 0;
    if (a.group) a.paths_per_block = std::max<int64_t>(a.paths_per_block, 4LL * kIntkWarps * a.group);
    a.X = X;
    a.M = M;
    a.F = F;
    a.cat = e->prep.has_cat ? 1 : 0;
    a.order = order;
    a.acc = acc;
    a.status = e->d_status;
    a.q = q;
    const size_t smem = intk_smem(F, a.sub, b.D).total;
    const int64_t blocks = ((b.n_paths + a.paths_per_block - 1) / a.paths_per_block) * a.n_tiles;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    switch (b.D) {
#define QTS_CASE(DD) \
    case DD: return launch_intk_d<DD>(a, blocks, smem, st);
        QTS_CASE(2) QTS_CASE(3) QTS_CASE(4) QTS_CASE(5) QTS_CASE(6) QTS_CASE(7) QTS_CASE(8) QTS_CASE(9)
        QTS_CASE(10) QTS_CASE(11) QTS_CASE(12) QTS_CASE(13) QTS_CASE(14) QTS_CASE(15) QTS_CASE(16)
#undef QTS_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qts

using namespace qts;

extern "C" qts_status qts_shap_interactions_order(qts_ensemble* e, const float* X, int64_t M, int32_t F,
                                                  int32_t order, int32_t n_quad, float* out,
                                                  qts_stream_t stream) {
    qts_status st = check_call(e, X, M, F, n_quad);
    if (st != QTS_OK) return st;
    if (order < 2 || order > kIntkMaxOrder)
        return fail(QTS_ERR_ARG, "order must be in [2, " + std::to_string(kIntkMaxOrder) + "]");
    if (M == 0) return QTS_OK;
    if (!out) return fail(QTS_ERR_ARG, "out is NULL");
    if (e->flags & QTS_FLAG_FP64)
        return fail(QTS_ERR_UNSUPPORTED, "interactions of order >= 2 by this entry point use the FP32 tables only");
    if (e->prep.max_unique > kIntkMaxD)
        return fail(QTS_ERR_UNSUPPORTED, "interactions of any order support paths of at most 16 unique features");
    const int64_t n_sub = binom_host(F, order);
    if (n_sub == 0) return QTS_OK;
    if (n_sub > ((int64_t)1 << 40) / std::max<int64_t>(M, 1))
        return fail(QTS_ERR_UNSUPPORTED, "C(F, order) * M is too large for the FP64 accumulators");
    cudaStream_t s = (cudaStream_t)stream;
    QuadF qf;  // QTS_NQ_EXACT: exact for the ensemble's widest path (this order, Thm 2)
    if (!make_quad(nodes_for(n_quad, e->prep.max_unique, order), &qf, nullptr))
        return fail(QTS_ERR_ARG, "quadrature rule");
    const size_t bytes = sizeof(double) * (size_t)(n_sub * M);
    st = ensure_workspace(e, bytes);
    if (st != QTS_OK) return st;
    double* acc = (double*)e->d_work;
    cudaError_t ce = cudaMemsetAsync(acc, 0, bytes, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "workspace clear");
    for (const Bucket& b : e->prep.buckets) {
        ce = launch_intk_bucket(e, b, X, M, F, order, qf, acc, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "order-s interaction kernel launch");
    }
    const int64_t n = n_sub * M;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8 * 152);
    intk_finalize_kernel<<<blocks, 256, 0, s>>>(acc, M, n_sub, out);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "order-s interaction finalize launch");
    return QTS_OK;
}

#endif  // QTS_HOST_PART
