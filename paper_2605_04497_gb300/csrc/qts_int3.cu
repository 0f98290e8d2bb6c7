// Third-order Shapley interaction indices (Thm 1 with |S| = 3; Alg. 1 with
// s = 3; exact for paths of at most 2 n + 2 unique features by Thm 2).
//
// For a path with elements sorted by feature and i < j < k,
//     SII_ijk += val d_i d_j d_k sum_m w_m prod_{l not in {i,j,k}} a_l(t_m),
// and the excluded product is P_i * prod_{i<l<j} a_l * prod_{j<l<k} a_l * S_k:
// two nested running products against the stored suffixes, no division.
// Triples are stored compactly (a < b < c, see tri3_index) and accumulated in
// FP64 in the workspace laid out [triple][sample] (one coalesced 256-byte add
// per warp and triple); a finalize kernel writes [sample][triple] in FP32.
//
// qts-build-parts: 5 (part 0: host code; parts 1-4: the per-width kernels)
#include <algorithm>
#include <string>

#include "qts_device.cuh"

namespace qts {

__host__ __device__ __forceinline__ int64_t choose2(int64_t n) { return n < 2 ? 0 : n * (n - 1) / 2; }
__host__ __device__ __forceinline__ int64_t choose3(int64_t n) { return n < 3 ? 0 : n * (n - 1) * (n - 2) / 6; }

// Index of the triple a < b < c < F: triples with a smaller first index, then
// pairs (b', c') of {a+1, ..} with b' < b, then c.
__host__ __device__ __forceinline__ int64_t tri3_index(int a, int b, int c, int F) {
    return (choose3(F) - choose3(F - a)) + (choose2(F - a - 1) - choose2(F - b)) + (c - b - 1);
}

struct Int3Args {
    const Rec32* rec;
    int64_t n_paths;
    int64_t paths_per_block;
    int sub;
    int n_tiles;
    const float* X;
    int64_t M;
    int F;
    int cat;            // ensemble has categorical elements: always the NaN-aware variant
    double* acc;        // [n_triples][M]
    int* status;
    QuadF q;
};

template <int D>
cudaError_t launch_int3_d(const Int3Args& a, int64_t blocks, size_t smem, cudaStream_t st);

#if QTS_DEVICE_PARTS

template <int D, int NP, bool HAS_NAN>
__device__ __forceinline__ void int3_path_f32(const Rec32* __restrict__ r, const float* __restrict__ xs,
                                              double* acc, int64_t s, int64_t M, int lane, int F,
                                              const QuadF& q) {
    constexpr int K = NP / 2;
    const float val = r[0].z;
    float dd[D];
    int nreal = D;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const Rec32 e = r[1 + j];
        const int f = feat_of(e.bits);
        const bool o = satisfies<HAS_NAN>(xs[f * kTileLd + lane], e.lo, e.hi, e.bits);
        dd[j] = (o ? 1.f : 0.f) - e.z;
        if (f >= F && j < nreal) nreal = j;
    }
    if (nreal < 3) return;
    const bool live = s < M;
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
#pragma unroll
        for (int i = 0; i < D - 2; ++i) {
            if (i + 2 >= nreal) break;
            const int fa = feat_of(r[1 + i].bits);
            float2 R1[K];
#pragma unroll
            for (int k = 0; k < K; ++k) R1[k] = P[i][k];
#pragma unroll
            for (int j = i + 1; j < D - 1; ++j) {
                if (j + 1 >= nreal) break;
                const int fb = feat_of(r[1 + j].bits);
                const int64_t base = tri3_index(fa, fb, fb + 1, F) - (fb + 1);  // + fc
                const float dij = dd[i] * dd[j];
                float2 R2[K];
#pragma unroll
                for (int k = 0; k < K; ++k) R2[k] = R1[k];
#pragma unroll
                for (int c = j + 1; c < D; ++c) {
                    if (c >= nreal) break;
                    float2 t = mul2(R2[0], S[c][0]);
#pragma unroll
                    for (int k = 1; k < K; ++k) t = fma2(R2[k], S[c][k], t);
                    if (c + 1 < D) {
#pragma unroll
                        for (int k = 0; k < K; ++k) R2[k] = mul2(R2[k], A[c][k]);
                    }
                    const float v = (t.x + t.y) * dij * dd[c];
                    if (live && v != 0.f)
                        atomicAdd(&acc[(base + feat_of(r[1 + c].bits)) * M + s], (double)v);
                }
#pragma unroll
                for (int k = 0; k < K; ++k) R1[k] = mul2(R1[k], A[j][k]);
            }
        }
    }
}

template <int D, int NP>
__global__ void __launch_bounds__(256) int3_kernel(Int3Args a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int F = a.F;
    float* xs = (float*)smem;
    size_t off = ((size_t)(F + 1) * kTileLd * 4 + 15) & ~(size_t)15;
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
    // The edge test is per element and the work per triple, so the NaN- and
    // category-aware test costs nothing measurable here: one variant serves all.
    (void)load_tile_t(xs, a.X, s0, a.M, F, F, 1);
    const int64_t s = s0 + lane;
    (void)stream_paths<Rec32, D>(a.rec, p0, p1, a.sub, st0, st1, bars, s_phase, &s_flag, a.status,
                                 [&](int64_t, const Rec32* r) {
                                     int3_path_f32<D, NP, true>(r, xs, a.acc, s, a.M, lane, F, a.q);
                                 });
}

template <int D>
cudaError_t launch_int3_d(const Int3Args& a, int64_t blocks, size_t smem, cudaStream_t st) {
    constexpr int NP = D <= 6 ? 8 : (D <= 12 ? 4 : 2);
    auto k = int3_kernel<D, NP>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)blocks, 128, smem, st>>>(a);
    return cudaGetLastError();
}


#define QTS_INST(DD) template cudaError_t launch_int3_d<DD>(const Int3Args&, int64_t, size_t, cudaStream_t);
#if QTS_IN_PART(1)
QTS_INST(16)
#endif
#if QTS_IN_PART(2)
QTS_INST(15)
#endif
#if QTS_IN_PART(3)
QTS_INST(14) QTS_INST(3) QTS_INST(4) QTS_INST(5) QTS_INST(6) QTS_INST(7) QTS_INST(8)
#endif
#if QTS_IN_PART(4)
QTS_INST(13) QTS_INST(9) QTS_INST(10) QTS_INST(11) QTS_INST(12)
#endif
#undef QTS_INST

#endif  // QTS_DEVICE_PARTS

#if !QTS_HOST_PART
}  // namespace qts
#endif

#if QTS_HOST_PART

size_t int3_smem_bytes(int F, int sub, int D) {
    size_t off = (size_t)(F + 1) * kTileLd * 4;
    off = (off + 15) & ~(size_t)15;
    off += 2 * (size_t)sub * (D + 1) * sizeof(Rec32);
    off = (off + 15) & ~(size_t)15;
    return off + 16;
}

// out[s][t] = acc[t][s] (FP64 -> FP32), one thread per (triple, sample).
__global__ void int3_finalize_kernel(const double* __restrict__ acc, int64_t M, int64_t n_tri,
                                     float* __restrict__ out) {
    const int64_t n = M * n_tri;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / M, s = i - t * M;
        out[s * n_tri + t] = (float)acc[i];
    }
}

static cudaError_t launch_int3_bucket(const qts_ensemble* e, const Bucket& b, const float* X, int64_t M, int F,
                                      const QuadF& q, double* acc, cudaStream_t st) {
    if (M <= 0 || b.n_paths == 0 || b.D < 3) return cudaSuccess;
    Int3Args a;
    a.rec = (const Rec32*)e->d_rec + b.rec_off;
    a.n_paths = b.n_paths;
    a.sub = 16;
    a.paths_per_block = 256;
    a.n_tiles = (int)((M + 31) / 32);
    a.X = X;
    a.M = M;
    a.F = F;
    a.cat = e->prep.has_cat ? 1 : 0;
    a.acc = acc;
    a.status = e->d_status;
    a.q = q;
    const size_t smem = int3_smem_bytes(F, a.sub, b.D);
    const int64_t blocks = ((b.n_paths + a.paths_per_block - 1) / a.paths_per_block) * a.n_tiles;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    switch (b.D) {
#define QTS_CASE(DD) \
    case DD: return launch_int3_d<DD>(a, blocks, smem, st);
        QTS_CASE(3) QTS_CASE(4) QTS_CASE(5) QTS_CASE(6) QTS_CASE(7) QTS_CASE(8) QTS_CASE(9) QTS_CASE(10)
        QTS_CASE(11) QTS_CASE(12) QTS_CASE(13) QTS_CASE(14) QTS_CASE(15) QTS_CASE(16)
#undef QTS_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qts

using namespace qts;

extern "C" qts_status qts_shap_interactions3(qts_ensemble* e, const float* X, int64_t M, int32_t F,
                                             int32_t n_quad, float* sii3, qts_stream_t stream) {
    qts_status st = check_call(e, X, M, F, n_quad);
    if (st != QTS_OK) return st;
    if (M == 0) return QTS_OK;
    if (!sii3) return fail(QTS_ERR_ARG, "sii3 is NULL");
    if (e->flags & QTS_FLAG_FP64)
        return fail(QTS_ERR_UNSUPPORTED, "third-order interactions use the FP32 tables only");
    if (e->prep.max_unique > 16)
        return fail(QTS_ERR_UNSUPPORTED, "third-order interactions support paths of at most 16 unique features");
    if (F > QTS_MAX_FEATURES_ORDER3)
        return fail(QTS_ERR_UNSUPPORTED, "third-order interactions support at most " +
                                             std::to_string(QTS_MAX_FEATURES_ORDER3) + " features");
    // few samples: the any-order kernel maps lanes to (path, sample) pairs and
    // writes the same compact layout
    if (M <= kFewRows) return qts_shap_interactions_order(e, X, M, F, 3, n_quad, sii3, stream);
    cudaStream_t s = (cudaStream_t)stream;
    QuadF qf;  // QTS_NQ_EXACT: exact for the ensemble's widest path (order 3, Thm 2)
    if (!make_quad(nodes_for(n_quad, e->prep.max_unique, 3), &qf, nullptr))
        return fail(QTS_ERR_ARG, "quadrature rule");
    const int64_t n_tri = choose3(F);
    if (n_tri == 0) return QTS_OK;
    const size_t bytes = sizeof(double) * (size_t)(n_tri * M);
    st = ensure_workspace(e, bytes);
    if (st != QTS_OK) return st;
    double* acc = (double*)e->d_work;
    cudaError_t ce = cudaMemsetAsync(acc, 0, bytes, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "workspace clear");
    for (const Bucket& b : e->prep.buckets) {
        ce = launch_int3_bucket(e, b, X, M, F, qf, acc, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "third-order kernel launch");
    }
    const int64_t n = n_tri * M;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8 * 152);
    int3_finalize_kernel<<<blocks, 256, 0, s>>>(acc, M, n_tri, sii3);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "third-order finalize launch");
    return QTS_OK;
}

#endif  // QTS_HOST_PART
