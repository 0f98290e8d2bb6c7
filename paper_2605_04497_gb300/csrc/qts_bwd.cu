// Adjoint of the first-order path (the paper has no adjoint; this
// differentiates Thm 1 / Eq. shap_as_weighted_banzhafs with the same n-point
// rule).  With L = sum_s sum_f grad_phi[s,f] phi[s,f], g_j = grad_phi[s, f_j],
// d_j = o_j - z_j, u_j = g_j d_j and a_j(t) = z_j + t d_j:
//
//   dL/dval   = sum_s sum_m w_m sum_i u_i prod_{l != i} a_l(t_m)
//   dL/dz_k   = sum_s val sum_m w_m [ -g_k prod_{l != k} a_l
//                                     + (1 - t_m) sum_{i != k} u_i prod_{l not in {i,k}} a_l ]
//
// (plus the bias terms of E[f], added in the epilogue).  Both are O(d) per
// (sample, path, node) with dual prefix products P_j = prod_{l<j} a_l,
// PU_j = sum_{i<j} u_i prod_{l<j, l != i} a_l and the matching suffixes S, SU:
//   prod_{l != k} a_l = P_k S_k,   sum_{i != k} u_i prod_{l != i,k} a_l = PU_k S_k + P_k SU_k.
// Products are recomputed per call, never stored.  Lanes are samples; the
// per-path sums over a tile of 32 samples are reduced in the warp and added to
// FP64 per-path / per-element accumulators, which an epilogue chains to the
// tree's edges:  dL/dw_e = dL/dz_k * prod_{other edges e' merged into k} w_e'.
//
// qts-build-parts: 6 (part 0: host code; parts 1-5: the per-width kernels)
#include <algorithm>
#include <type_traits>

#include "qts_paths.cuh"

namespace qts {

struct BwdArgs {
    const void* rec;
    int64_t n_paths;
    int64_t paths_per_block;
    int sub;
    int n_tiles;
    const float* X;
    const float* G;     // grad_phi, M x (F+1)
    int64_t M;
    int F;
    int cat;            // ensemble has categorical elements: always the NaN-aware variant
    double* g_val;      // per path of this bucket
    double* g_slot;     // per element slot of this bucket (n_paths * D)
    double* phi;        // fused forward output (M x (F+1)) or nullptr
    int* status;
    QuadF q;
    QuadD qd;
};

template <int D>
cudaError_t launch_bwd_d(const BwdArgs& a, int np, bool fp64, bool with_phi, int warps, int64_t blocks,
                         size_t smem, cudaStream_t st);

#if QTS_DEVICE_PARTS

// --------------------------------------------------------------- kernel ---

template <typename Rec, typename Acc>
__device__ __forceinline__ void bwd_smem_layout(int F, int sub, int D, bool with_phi, float** xs,
                                                float** gs, Acc** ps, Rec** st0, Rec** st1,
                                                uint64_t** bars, unsigned char* base) {
    const size_t rows = F + 1;
    size_t off = 0;
    *xs = (float*)(base + off);
    off += rows * kTileLd * sizeof(float);
    *gs = (float*)(base + off);
    off += rows * kTileLd * sizeof(float);
    off = (off + 15) & ~(size_t)15;
    *ps = (Acc*)(base + off);
    if (with_phi) off += rows * kTileLd * sizeof(Acc);
    off = (off + 15) & ~(size_t)15;
    *st0 = (Rec*)(base + off);
    off += (size_t)sub * (D + 1) * sizeof(Rec);
    *st1 = (Rec*)(base + off);
    off += (size_t)sub * (D + 1) * sizeof(Rec);
    off = (off + 15) & ~(size_t)15;
    *bars = (uint64_t*)(base + off);
}

template <int D, int NP, bool FP64, bool WITH_PHI>
__global__ void __launch_bounds__(256) bwd_kernel(BwdArgs a) {
    using Rec = typename std::conditional<FP64, Rec64, Rec32>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    float *xs, *gs, *ps;
    Rec *st0, *st1;
    uint64_t* bars;
    bwd_smem_layout<Rec, float>(a.F, a.sub, D, WITH_PHI, &xs, &gs, &ps, &st0, &st1, &bars, smem);
    __shared__ int s_flag;
    __shared__ uint32_t s_phase[2];

    const int F = a.F;
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
    if (WITH_PHI)
        for (int idx = threadIdx.x; idx < (F + 1) * kTileLd; idx += blockDim.x) ps[idx] = 0.f;
    const bool has_nan = load_tile_t(xs, a.X, s0, a.M, F, F, 1) || a.cat != 0;
    // grad_phi tile: columns 0..F-1 (column F, the bias weight, is handled in
    // the epilogue); row F stays zero for padding elements
    load_tile_t(gs, a.G, s0, a.M, F, F + 1, 1);

    const bool ok = stream_paths<Rec, D>(
        (const Rec*)a.rec, p0, p1, a.sub, st0, st1, bars, s_phase, &s_flag, a.status,
        [&](int64_t p, const Rec* r) {
            double* gsl = a.g_slot + p * D;
            double* gv = a.g_val + (FP64 ? p : 2 * p);  // FP32: pair tables, two sums per path
            if constexpr (FP64) {
                if (has_nan) bwd_path_f64<D, true>(r, xs, gs, lane, a.qd, gsl, gv);
                else bwd_path_f64<D, false>(r, xs, gs, lane, a.qd, gsl, gv);
            } else {
                const SmemCols xr{xs, lane}, gr{gs, lane};
                if constexpr (D <= 16) {
                    if (has_nan) bwd_path_f32_pk<D, true, WITH_PHI ? kPhiAtomic : kPhiNone, SmemCols, SmemCols, true>(r, xr, gr, ps, lane, a.q, gsl, gv);
                    else bwd_path_f32_pk<D, false, WITH_PHI ? kPhiAtomic : kPhiNone, SmemCols, SmemCols, true>(r, xr, gr, ps, lane, a.q, gsl, gv);
                } else {
                    if (has_nan) bwd_path_f32<D, NP, true, WITH_PHI ? kPhiAtomic : kPhiNone, false, SmemCols, SmemCols, true>(r, xr, gr, ps, lane, a.q, gsl, gv);
                    else bwd_path_f32<D, NP, false, WITH_PHI ? kPhiAtomic : kPhiNone, false, SmemCols, SmemCols, true>(r, xr, gr, ps, lane, a.q, gsl, gv);
                }
            }
        });
    if (!ok) return;
    if (WITH_PHI) {
        for (int idx = threadIdx.x; idx < 32 * F; idx += blockDim.x) {
            const int s = idx / F, f = idx - s * F;
            if (s0 + s < a.M) {
                const float v = ps[f * kTileLd + s];
                if (v != 0.f) atomicAdd(&a.phi[(s0 + s) * (F + 1) + f], (double)v);
            }
        }
    }
}

// ---------------------------------------------------------- launchers -----

template <int D, int NP, bool FP64, bool WP>
static cudaError_t launch_bwd_t(const BwdArgs& a, int warps, int64_t blocks, size_t smem, cudaStream_t st) {
    auto k = bwd_kernel<D, NP, FP64, WP>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)blocks, warps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_bwd_d(const BwdArgs& a, int np, bool fp64, bool with_phi, int warps,
                                int64_t blocks, size_t smem, cudaStream_t st) {
    if (fp64) return launch_bwd_t<D, 2, true, false>(a, warps, blocks, smem, st);
    if constexpr (D <= 8) {
        if (np >= 4) {
            if (with_phi) return launch_bwd_t<D, 4, false, true>(a, warps, blocks, smem, st);
            return launch_bwd_t<D, 4, false, false>(a, warps, blocks, smem, st);
        }
    }
    if (with_phi) return launch_bwd_t<D, 2, false, true>(a, warps, blocks, smem, st);
    return launch_bwd_t<D, 2, false, false>(a, warps, blocks, smem, st);
}

#define QTS_INST(DD) \
    template cudaError_t launch_bwd_d<DD>(const BwdArgs&, int, bool, bool, int, int64_t, size_t, cudaStream_t);
#if QTS_IN_PART(1)
QTS_INST(64)
#endif
#if QTS_IN_PART(2)
QTS_INST(56)
#endif
#if QTS_IN_PART(3)
QTS_INST(48) QTS_INST(40)
#endif
#if QTS_IN_PART(4)
QTS_INST(32) QTS_INST(28) QTS_INST(24) QTS_INST(20)
#endif
#if QTS_IN_PART(5)
QTS_INST(1) QTS_INST(2) QTS_INST(3) QTS_INST(4) QTS_INST(5) QTS_INST(6) QTS_INST(7) QTS_INST(8) QTS_INST(9) QTS_INST(10) QTS_INST(11) QTS_INST(12) QTS_INST(13) QTS_INST(14) QTS_INST(15) QTS_INST(16)
#endif
#undef QTS_INST

#endif  // QTS_DEVICE_PARTS

#if !QTS_HOST_PART
}  // namespace qts
#endif

#if QTS_HOST_PART

size_t bwd_smem_bytes(int F, int sub, int D, bool fp64, bool with_phi) {
    const size_t rows = F + 1;
    size_t off = 2 * rows * kTileLd * 4;
    off = (off + 15) & ~(size_t)15;
    if (with_phi) off += rows * kTileLd * (fp64 ? 8 : 4);
    off = (off + 15) & ~(size_t)15;
    off += 2 * (size_t)sub * (D + 1) * (fp64 ? sizeof(Rec64) : sizeof(Rec32));
    off = (off + 15) & ~(size_t)15;
    return off + 16;
}

// ------------------------------------------------------------ epilogue ----

// G = sum_s grad_phi[s, F]  (the weight of E[f] in L), FP64.
__global__ void bias_grad_kernel(const float* __restrict__ G, int64_t M, int F, double* out) {
    double acc = 0.0;
    for (int64_t s = threadIdx.x; s < M; s += blockDim.x) acc += (double)G[s * (F + 1) + F];
    for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *out = t;
    }
}

// d_leaf of every path's leaf: sum over samples + bias term G * prod_j z_j;
// single-leaf trees contribute G (their value is part of E[f] directly).
__global__ void path_epilogue_kernel(int64_t n_paths, const int64_t* __restrict__ leaf,
                                     const double* __restrict__ zprod, const double* __restrict__ g_val,
                                     const double* __restrict__ gb, int64_t n_empty,
                                     const int64_t* __restrict__ empty_leaf, double* d_leaf) {
    const double G = *gb;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_paths + n_empty;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (p < n_paths) d_leaf[leaf[p]] = g_val[p] + G * zprod[p];
        else d_leaf[empty_leaf[p - n_paths]] = G;
    }
}

struct SlotMap {
    int nb;
    int64_t slot_base[kMaxBuckets + 1];
    int64_t path_base[kMaxBuckets];
    int D[kMaxBuckets];
};

// Chain each element's dL/dz to the edges merged into it.
__global__ void slot_epilogue_kernel(SlotMap sm, const double* __restrict__ g_slot,
                                     const double* __restrict__ path_val,
                                     const double* __restrict__ zexcl, const int64_t* __restrict__ eb,
                                     const int64_t* __restrict__ enode, const double* __restrict__ ecoef,
                                     const double* __restrict__ gb, double* d_z) {
    const double G = *gb;
    const int64_t n_slots = sm.slot_base[sm.nb];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_slots;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = eb[s], e1 = eb[s + 1];
        if (e0 == e1) continue;  // padding slot
        int b = 0;
        while (b + 1 < sm.nb && s >= sm.slot_base[b + 1]) ++b;
        const int64_t p = sm.path_base[b] + (s - sm.slot_base[b]) / sm.D[b];
        const double tot = g_slot[s] + G * path_val[p] * zexcl[s];
        for (int64_t e = e0; e < e1; ++e) atomicAdd(&d_z[enode[e]], tot * ecoef[e]);
    }
}

cudaError_t launch_bwd_bucket(const qts_ensemble* e, const Bucket& b, const float* X,
                              const float* grad, int64_t M, int F, const QuadF& q, double* g_val,
                              double* g_slot, double* phi, const Tune& tn, cudaStream_t st) {
    if (M <= 0 || b.n_paths == 0) return cudaSuccess;
    const bool fp64 = (e->flags & QTS_FLAG_FP64) != 0;
    QuadD qd;
    make_quad(q.n, nullptr, &qd, 2);
    BwdArgs a;
    // FP32: the pair tables (two adjoint sums per path), FP64: the per-leaf tables
    a.rec = fp64 ? (const void*)((const Rec64*)e->d_rec + b.rec_off)
                 : (const void*)((const Rec32*)e->bdev.rec + b.rec_off);
    a.n_paths = b.n_paths;
    const bool with_phi = phi != nullptr && !fp64;
    a.sub = std::max(1, tn.sub);
    // wide inputs: stage fewer paths at a time until the block fits shared memory
    while (a.sub > 1 && bwd_smem_bytes(F, a.sub, b.D, fp64, with_phi) > kSmemMax) a.sub /= 2;
    a.paths_per_block = std::max<int64_t>(a.sub, (int64_t)tn.paths / a.sub * a.sub);
    a.n_tiles = (int)((M + 31) / 32);
    a.X = X;
    a.G = grad;
    a.M = M;
    a.F = F;
    a.cat = (fp64 ? e->prep.has_cat : e->bprep.has_cat) ? 1 : 0;
    a.g_val = g_val + (fp64 ? 1 : 2) * b.path_base;
    a.g_slot = g_slot + b.slot_base;
    a.phi = phi;
    a.status = e->d_status;
    a.q = q;
    a.qd = qd;
    const int64_t chunks = (b.n_paths + a.paths_per_block - 1) / a.paths_per_block;
    const int64_t blocks = chunks * a.n_tiles;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const size_t smem = bwd_smem_bytes(F, a.sub, b.D, fp64, with_phi);
    if (smem > kSmemMax) return cudaErrorInvalidConfiguration;
    const int warps = std::max(1, std::min(8, tn.warps));
    // nodes per register pass; it must divide the rule's padded node count
    const int np = (b.D <= 8 && q.n_pad % 4 == 0) ? 4 : 2;
    if (q.n_pad % 2 != 0) return cudaErrorInvalidValue;
    switch (b.D) {
#define QTS_CASE(DD) \
    case DD: return launch_bwd_d<DD>(a, np, fp64, with_phi, warps, blocks, smem, st);
        QTS_CASE(1) QTS_CASE(2) QTS_CASE(3) QTS_CASE(4) QTS_CASE(5) QTS_CASE(6) QTS_CASE(7)
        QTS_CASE(8) QTS_CASE(9) QTS_CASE(10) QTS_CASE(11) QTS_CASE(12) QTS_CASE(13) QTS_CASE(14)
        QTS_CASE(15) QTS_CASE(16) QTS_CASE(20) QTS_CASE(24) QTS_CASE(28) QTS_CASE(32)
        QTS_CASE(40) QTS_CASE(48) QTS_CASE(56) QTS_CASE(64)
#undef QTS_CASE
        default: return cudaErrorInvalidValue;
    }
}

// Pair tables: d_leaf of each path's leaf, and of leaf B of a sibling pair.
// The kernel leaves sum_s o_A K and sum_s o_B K in g_val[2p], g_val[2p + 1]
// (o K = the leaf's share of the pair element's adjoint); dL/dval_k adds
// z_k * Q with Q the pair element's slot sum, and the bias term G prod z.
__global__ void pair_path_epilogue_kernel(int64_t n_paths, const int64_t* __restrict__ leaf,
                                          const double* __restrict__ zprod, const int64_t* __restrict__ leaf2,
                                          const double* __restrict__ zprod2, const double* __restrict__ pz,
                                          const int64_t* __restrict__ gslot, const double* __restrict__ g_val,
                                          const double* __restrict__ g_slot, const double* __restrict__ gb,
                                          int64_t n_empty, const int64_t* __restrict__ empty_leaf, double* d_leaf) {
    const double G = *gb;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_paths + n_empty;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (p >= n_paths) {
            d_leaf[empty_leaf[p - n_paths]] = G;
            continue;
        }
        const int64_t l2 = leaf2[p];
        if (l2 < 0) {
            d_leaf[leaf[p]] = g_val[2 * p] + G * zprod[p];
        } else {
            const double Q = g_slot[gslot[p]];
            d_leaf[leaf[p]] = pz[2 * p] * Q + g_val[2 * p] + G * zprod[p];
            d_leaf[l2] = pz[2 * p + 1] * Q + g_val[2 * p + 1] + G * zprod2[p];
        }
    }
}

static SlotMap slot_map(const Prepared& P) {
    SlotMap sm;
    sm.nb = (int)P.buckets.size();
    for (int b = 0; b < sm.nb; ++b) {
        sm.slot_base[b] = P.buckets[b].slot_base;
        sm.path_base[b] = P.buckets[b].path_base;
        sm.D[b] = P.buckets[b].D;
    }
    sm.slot_base[sm.nb] = P.n_slots;
    return sm;
}

cudaError_t launch_bwd_epilogue_pairs(const qts_ensemble* e, const float* grad, int64_t M, int F,
                                      const double* g_val, const double* g_slot, double* d_leaf,
                                      double* d_z, double* gb, cudaStream_t st) {
    const Prepared& P = e->bprep;
    const DevTables& T = e->bdev;
    cudaError_t err = cudaMemsetAsync(d_leaf, 0, sizeof(double) * e->n_nodes, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(d_z, 0, sizeof(double) * e->n_nodes, st);
    if (err != cudaSuccess) return err;
    bias_grad_kernel<<<1, 1024, 0, st>>>(grad, M, F, gb);
    const int64_t np = P.n_paths + (int64_t)P.empty_leaf.size();
    if (np > 0) {
        const int blocks = (int)std::min<int64_t>((np + 255) / 256, 8 * 152);
        pair_path_epilogue_kernel<<<blocks, 256, 0, st>>>(P.n_paths, T.path_leaf, T.path_zprod, T.pair_leaf2,
                                                          T.pair_zprod2, T.pair_z, T.pair_gslot, g_val, g_slot, gb,
                                                          (int64_t)P.empty_leaf.size(), T.empty_leaf, d_leaf);
    }
    if (P.n_slots > 0) {
        const int blocks = (int)std::min<int64_t>((P.n_slots + 255) / 256, 8 * 152);
        slot_epilogue_kernel<<<blocks, 256, 0, st>>>(slot_map(P), g_slot, T.path_val, T.slot_zexcl,
                                                     T.slot_edge_begin, T.edge_node, T.edge_coef, gb, d_z);
    }
    return cudaGetLastError();
}

cudaError_t launch_bwd_epilogue(const qts_ensemble* e, const float* grad, int64_t M, int F,
                                const double* g_val, const double* g_slot, double* d_leaf,
                                double* d_z, double* gb, cudaStream_t st) {
    const Prepared& P = e->prep;
    cudaError_t err = cudaMemsetAsync(d_leaf, 0, sizeof(double) * e->n_nodes, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(d_z, 0, sizeof(double) * e->n_nodes, st);
    if (err != cudaSuccess) return err;
    bias_grad_kernel<<<1, 1024, 0, st>>>(grad, M, F, gb);
    const int64_t np = P.n_paths + (int64_t)P.empty_leaf.size();
    if (np > 0) {
        const int blocks = (int)std::min<int64_t>((np + 255) / 256, 8 * 152);
        path_epilogue_kernel<<<blocks, 256, 0, st>>>(P.n_paths, e->d_path_leaf, e->d_path_zprod,
                                                     g_val, gb, (int64_t)P.empty_leaf.size(),
                                                     e->d_empty_leaf, d_leaf);
    }
    if (P.n_slots > 0) {
        SlotMap sm;
        sm.nb = (int)P.buckets.size();
        for (int b = 0; b < sm.nb; ++b) {
            sm.slot_base[b] = P.buckets[b].slot_base;
            sm.path_base[b] = P.buckets[b].path_base;
            sm.D[b] = P.buckets[b].D;
        }
        sm.slot_base[sm.nb] = P.n_slots;
        const int blocks = (int)std::min<int64_t>((P.n_slots + 255) / 256, 8 * 152);
        slot_epilogue_kernel<<<blocks, 256, 0, st>>>(sm, g_slot, e->d_path_val, e->d_slot_zexcl,
                                                     e->d_slot_edge_begin, e->d_edge_node,
                                                     e->d_edge_coef, gb, d_z);
    }
    return cudaGetLastError();
}

}  // namespace qts

using namespace qts;

extern "C" qts_status qts_shap_backward(qts_ensemble* e, const float* X, int64_t M, int32_t F,
                                        int32_t n_quad, const float* grad_phi, double* d_leaf,
                                        double* d_z, qts_stream_t stream) {
    qts_status st = check_call(e, X, M, F, n_quad);
    if (st != QTS_OK) return st;
    if (!d_leaf || !d_z) return fail(QTS_ERR_ARG, "d_leaf and d_z must be non-NULL");
    if (M > 0 && !grad_phi) return fail(QTS_ERR_ARG, "grad_phi is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    // FP32 runs on the pair tables (two sums per path), FP64 on the per-leaf tables
    const bool fp64 = (e->flags & QTS_FLAG_FP64) != 0;
    if (!fp64) {
        st = ensure_batch_tables(e);
        if (st != QTS_OK) return st;
    }
    const Prepared& P = fp64 ? e->prep : e->bprep;
    const int per_path = fp64 ? 1 : 2;
    const size_t bytes = sizeof(double) * (size_t)(4 + per_path * P.n_paths + P.n_slots);
    st = ensure_workspace(e, bytes);
    if (st != QTS_OK) return st;
    double* gb = (double*)e->d_work;
    double* g_val = gb + 4;
    double* g_slot = g_val + per_path * P.n_paths;
    cudaError_t ce = cudaMemsetAsync(e->d_work, 0, bytes, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "workspace clear");
    if (M > 0) {
        for (const Bucket& b : P.buckets) {
            // the bucket's rule, padded to whole node pairs (QTS_NQ_EXACT: ceil(D/2) points)
            QuadF qf;
            if (!make_quad(nodes_for(n_quad, b.D, 1), &qf, nullptr, 2)) return fail(QTS_ERR_ARG, "quadrature rule");
            ce = launch_bwd_bucket(e, b, X, grad_phi, M, F, qf, g_val, g_slot, nullptr, e->tune[b.D], s);
            if (ce != cudaSuccess) return cuda_fail(ce, "adjoint kernel launch");
        }
        ce = fp64 ? launch_bwd_epilogue(e, grad_phi, M, F, g_val, g_slot, d_leaf, d_z, gb, s)
                  : launch_bwd_epilogue_pairs(e, grad_phi, M, F, g_val, g_slot, d_leaf, d_z, gb, s);
    } else {
        ce = cudaMemsetAsync(d_leaf, 0, sizeof(double) * e->n_nodes, s);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(d_z, 0, sizeof(double) * e->n_nodes, s);
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "adjoint epilogue");
    return QTS_OK;
}

#endif  // QTS_HOST_PART
