// First-order Shapley values (Thm 1 with S = {i}, Eq. shap_as_weighted_banzhafs).
//
// Work decomposition: a block owns a tile of 32 samples (lane = sample) and a
// chunk of paths of one bucket (all paths have D merged elements).  Its warps
// take the chunk's paths round-robin; every lane evaluates, for its sample,
//     c_i = sum_m w_m val prod_{j<i} a_j(t_m) prod_{j>i} a_j(t_m),
//     a_j(t) = z_j + t (o_j - z_j),
// by a prefix product (seeded with w_m * val) and a suffix product - no
// division - with two quadrature nodes packed per f32x2 register pair, and
// adds (o_i - z_i) c_i to phi[s, f_i] in a shared FP32 tile.  Path records are
// staged in shared memory by bulk (TMA) copies, double-buffered; the FP32 tile
// is flushed into the FP64 output with atomics once per block.
//
// qts-build-parts: 6 (part 0: host code; parts 1-5: the per-width kernels)
#include <algorithm>
#include <type_traits>

#include "qts_paths.cuh"

namespace qts {

struct FwdArgs {
    const void* rec;    // bucket records (Rec32 or Rec64)
    int64_t n_paths;
    int64_t paths_per_block;
    int sub;            // paths per staged sub-chunk
    int n_tiles;        // sample tiles of 32
    const float* X;
    int64_t M;
    int F;
    int cat;            // ensemble has categorical elements: always the NaN-aware variant
    double* phi;        // M x (F+1)
    int* status;
    int ntiles;         // sample tiles of 32 per block: 1 (warps share the tile and
                        // split paths, atomics) or the warp count (each warp owns a
                        // tile and walks every path; private phi tile, no atomics)
    int gphi;           // FP64 only: 1 = no accumulator tile (it would not fit shared
                        // memory), contributions go straight to phi with FP64 atomics
    int group;          // few samples (M <= 16): lanes are (path, sample) pairs, a warp
                        // takes `group` = 32 / M paths at a time (FP32 only); 0 otherwise
    int nphi;           // phi tiles: ntiles, or (FP32, ntiles = 1) one per warp, when the
                        // warps share a sample tile, split the paths and each add into
                        // its own phi tile (no atomics; summed at the flush)
    QuadF q;
    QuadD qd;
};

template <int D>
cudaError_t launch_fwd_d(const FwdArgs& a, int np, bool fp64, int warps, int64_t blocks, size_t smem,
                         cudaStream_t st);

#if QTS_DEVICE_PARTS

// --------------------------------------------------------------- kernel ---

template <typename Rec, typename Acc>
__device__ __forceinline__ size_t fwd_smem_layout(int F, int sub, int D, int ntiles, int nphi, bool gphi,
                                                  float** xs, Acc** ps, Rec** stage0, Rec** stage1,
                                                  uint64_t** bars, unsigned char* base) {
    const int rows = F + 1;
    size_t off = 0;
    *xs = (float*)(base + off);
    off += (size_t)ntiles * rows * kTileLd * sizeof(float);
    off = (off + 15) & ~(size_t)15;
    *ps = (Acc*)(base + off);
    if (!gphi) off += (size_t)nphi * rows * kTileLd * sizeof(Acc);
    off = (off + 15) & ~(size_t)15;
    *stage0 = (Rec*)(base + off);
    off += (size_t)sub * (D + 1) * sizeof(Rec);
    *stage1 = (Rec*)(base + off);
    off += (size_t)sub * (D + 1) * sizeof(Rec);
    off = (off + 15) & ~(size_t)15;
    *bars = (uint64_t*)(base + off);
    off += 2 * sizeof(uint64_t);
    return off;
}

template <int D, int NP, bool FP64>
__global__ void __launch_bounds__(256) fwd_kernel(FwdArgs a) {
    using Rec = typename std::conditional<FP64, Rec64, Rec32>::type;
    using Acc = typename std::conditional<FP64, double, float>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    float* xs;
    Acc* ps;
    Rec *st0, *st1;
    uint64_t* bars;
    fwd_smem_layout<Rec, Acc>(a.F, a.sub, D, a.ntiles, a.nphi, a.gphi != 0, &xs, &ps, &st0, &st1, &bars, smem);
    __shared__ int s_flag;
    __shared__ uint32_t s_phase[2];

    const int F = a.F;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool priv = a.ntiles > 1;   // each warp its own samples and phi tile
    const bool own = a.nphi > 1;      // each warp its own phi tile (priv, or split paths)
    const int stride = (F + 1) * kTileLd;
    const int group = (int)(blockIdx.x % (unsigned)a.n_tiles);
    const int64_t chunk = blockIdx.x / (unsigned)a.n_tiles;
    const int64_t s0 = (int64_t)group * 32 * a.ntiles;
    const int64_t p0 = chunk * a.paths_per_block;
    const int64_t p1 = imin64(p0 + a.paths_per_block, a.n_paths);
    float* my_xs = priv ? xs + warp * stride : xs;
    Acc* my_ps = own ? ps + warp * stride : ps;
    const int64_t sw = priv ? s0 + 32 * warp : s0;

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
        s_phase[0] = s_phase[1] = 0;
    }
    if (!a.gphi)
        for (int idx = threadIdx.x; idx < a.nphi * stride; idx += blockDim.x) ps[idx] = (Acc)0;
    // sample tiles (row = feature, column = sample) plus a zero row F for padding
    const bool has_nan = load_tiles_t(xs, a.X, s0, a.M, F, F, 1, a.ntiles, stride) || a.cat != 0;

    bool ok;
    if (!FP64 && a.group > 0) {
        // few samples: lane (slot, sample) evaluates path slot of each group for
        // its sample (column of the tile); the shared phi tile takes atomics
        const int slot = lane / (int)a.M, col = lane - slot * (int)a.M;
        walk_paths_grouped<Rec, D>((const Rec*)a.rec, p0, p1, a.group, slot, [&](int64_t, const Rec* r, bool valid) {
            if constexpr (!FP64) {
                if (!valid) return;
                const SmemCols xr{xs, col};
                if (has_nan) fwd_path_f32<D, NP, true, SmemCols, kPhiAtomic, true>(r, xr, ps, col, a.q);
                else fwd_path_f32<D, NP, false, SmemCols, kPhiAtomic, true>(r, xr, ps, col, a.q);
            }
        });
        ok = true;
        __syncthreads();  // every warp's adds are in the tile before the flush
    } else {
    ok = stream_paths<Rec, D>(
        (const Rec*)a.rec, p0, p1, a.sub, st0, st1, bars, s_phase, &s_flag, a.status,
        [&](int64_t, const Rec* r) {
            if constexpr (FP64) {
                if (a.gphi) {
                    // this lane's row of phi (lanes past M only skip their adds)
                    const bool live = sw + lane < a.M;
                    double* row = a.phi + (live ? (sw + lane) * (F + 1) : 0);
                    if (has_nan) fwd_path_f64<D, true>(r, my_xs, row, lane, a.qd, F, live);
                    else fwd_path_f64<D, false>(r, my_xs, row, lane, a.qd, F, live);
                } else {
                    if (has_nan) fwd_path_f64<D, true>(r, my_xs, my_ps, lane, a.qd);
                    else fwd_path_f64<D, false>(r, my_xs, my_ps, lane, a.qd);
                }
            } else {
                const SmemCols xr{my_xs, lane};
                if (own) {
                    if (has_nan) fwd_path_f32<D, NP, true, SmemCols, kPhiPrivate, true>(r, xr, my_ps, lane, a.q);
                    else fwd_path_f32<D, NP, false, SmemCols, kPhiPrivate, true>(r, xr, my_ps, lane, a.q);
                } else {
                    if (has_nan) fwd_path_f32<D, NP, true, SmemCols, kPhiAtomic, true>(r, xr, my_ps, lane, a.q);
                    else fwd_path_f32<D, NP, false, SmemCols, kPhiAtomic, true>(r, xr, my_ps, lane, a.q);
                }
            }
        },
        priv);
    }
    if (!ok || a.gphi) return;
    const int nflush = 32 * F;
    if (priv) {
        for (int idx = lane; idx < nflush; idx += 32) {
            const int s = idx / F, f = idx - s * F;
            if (sw + s < a.M) {
                const Acc v = my_ps[f * kTileLd + s];
                if (v != (Acc)0) atomicAdd(&a.phi[(sw + s) * (F + 1) + f], (double)v);
            }
        }
    } else if (own) {
        // stream_paths ended on a block barrier: every warp's tile is complete
        for (int idx = threadIdx.x; idx < nflush; idx += blockDim.x) {
            const int s = idx / F, f = idx - s * F;
            if (s0 + s < a.M) {
                Acc v = (Acc)0;
                for (int w = 0; w < a.nphi; ++w) v += ps[w * stride + f * kTileLd + s];
                if (v != (Acc)0) atomicAdd(&a.phi[(s0 + s) * (F + 1) + f], (double)v);
            }
        }
    } else {
        for (int idx = threadIdx.x; idx < nflush; idx += blockDim.x) {
            const int s = idx / F, f = idx - s * F;
            if (s0 + s < a.M) {
                const Acc v = ps[f * kTileLd + s];
                if (v != (Acc)0) atomicAdd(&a.phi[(s0 + s) * (F + 1) + f], (double)v);
            }
        }
    }
}

// ---------------------------------------------------------- dispatch ------

template <int D, int NP, bool FP64>
static cudaError_t launch_fwd_t(const FwdArgs& a, int warps, int64_t blocks, size_t smem,
                                cudaStream_t st) {
    auto k = fwd_kernel<D, NP, FP64>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)blocks, warps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_fwd_d(const FwdArgs& a, int np, bool fp64, int warps, int64_t blocks, size_t smem,
                         cudaStream_t st) {
    if (fp64) return launch_fwd_t<D, 2, true>(a, warps, blocks, smem, st);
    if constexpr (D <= 8) {
        if (np >= 8) return launch_fwd_t<D, 8, false>(a, warps, blocks, smem, st);
    }
    if constexpr (D <= 24) {
        if (np >= 4) return launch_fwd_t<D, 4, false>(a, warps, blocks, smem, st);
    }
    return launch_fwd_t<D, 2, false>(a, warps, blocks, smem, st);
}

#define QTS_INST(DD) \
    template cudaError_t launch_fwd_d<DD>(const FwdArgs&, int, bool, int, int64_t, size_t, cudaStream_t);
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
QTS_INST(1) QTS_INST(2) QTS_INST(3) QTS_INST(4) QTS_INST(5) QTS_INST(6) QTS_INST(7) QTS_INST(8)
QTS_INST(9) QTS_INST(10) QTS_INST(11) QTS_INST(12) QTS_INST(13) QTS_INST(14) QTS_INST(15) QTS_INST(16)
#endif
#undef QTS_INST

#endif  // QTS_DEVICE_PARTS

#if !QTS_HOST_PART
}  // namespace qts
#endif

#if QTS_HOST_PART

// phi[:, :F] = 0, phi[:, F] = E[f]
__global__ void phi_init_kernel(double* phi, int64_t M, int F, double bias) {
    const int64_t n = M * (F + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        phi[i] = (i % (F + 1) == F) ? bias : 0.0;
}

cudaError_t launch_phi_init(double* phi, int64_t M, int F, double bias, cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    const int64_t n = M * (F + 1);
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4 * 152);
    phi_init_kernel<<<blocks, 256, 0, st>>>(phi, M, F, bias);
    return cudaGetLastError();
}

size_t fwd_smem_bytes(int F, int sub, int D, bool fp64, int ntiles, bool gphi = false, int nphi = 0) {
    const size_t rows = F + 1;
    size_t off = ntiles * rows * kTileLd * 4;
    off = (off + 15) & ~(size_t)15;
    if (!gphi) off += (nphi > 0 ? nphi : ntiles) * rows * kTileLd * (fp64 ? 8 : 4);
    off = (off + 15) & ~(size_t)15;
    off += 2 * (size_t)sub * (D + 1) * (fp64 ? sizeof(Rec64) : sizeof(Rec32));
    off = (off + 15) & ~(size_t)15;
    return off + 16;
}

cudaError_t launch_fwd_bucket(const qts_ensemble* e, const Bucket& b, const float* X, int64_t M,
                              int F, const QuadF& q, const QuadD& qd, double* phi, const Tune& tn,
                              cudaStream_t st) {
    if (M <= 0 || b.n_paths == 0) return cudaSuccess;
    const bool fp64 = (e->flags & QTS_FLAG_FP64) != 0;
    FwdArgs a;
    // FP32: the pair tables (sibling leaves merged), whose buckets the caller walks
    a.rec = fp64 ? (const void*)((const Rec64*)e->d_rec + b.rec_off)
                 : (const void*)((const Rec32*)e->bdev.rec + b.rec_off);
    a.n_paths = b.n_paths;
    a.sub = std::max(1, tn.sub);
    const int warps = std::max(1, std::min(8, tn.warps));
    // tn.priv 1: each warp its own 32 samples and tiles, when they stay small;
    // 2: the warps share 32 samples, split the paths, a phi tile each; 0: the
    // warps share 32 samples and one phi tile (shared-memory atomics)
    a.ntiles = (!fp64 && tn.priv == 1 && fwd_smem_bytes(F, a.sub, b.D, false, warps) <= 100 * 1024) ? warps : 1;
    a.group = (!fp64 && M <= kFewRows) ? (int)(32 / M) : 0;
    if (a.group) a.ntiles = 1;
    a.nphi = (!fp64 && !a.group && tn.priv == 2 && warps > 1 &&
              fwd_smem_bytes(F, a.sub, b.D, false, 1, false, warps) <= 100 * 1024) ? warps : a.ntiles;
    // wide inputs: stage fewer paths at a time, and (FP64) drop the accumulator
    // tile for direct FP64 atomics into phi, until the block fits shared memory
    a.gphi = 0;
    while (a.sub > 1 && fwd_smem_bytes(F, a.sub, b.D, fp64, a.ntiles, false, a.nphi) > kSmemMax) a.sub /= 2;
    if (fp64 && fwd_smem_bytes(F, a.sub, b.D, fp64, a.ntiles) > kSmemMax) {
        a.gphi = 1;
        a.sub = std::max(1, tn.sub);
        while (a.sub > 1 && fwd_smem_bytes(F, a.sub, b.D, fp64, a.ntiles, true) > kSmemMax) a.sub /= 2;
    }
    a.paths_per_block = std::max<int64_t>(a.sub, (int64_t)tn.paths / a.sub * a.sub);
    if (a.group) a.paths_per_block = std::max<int64_t>(a.paths_per_block, 4LL * warps * a.group);
    a.n_tiles = (int)((M + 32 * a.ntiles - 1) / (32 * a.ntiles));
    a.X = X;
    a.M = M;
    a.F = F;
    a.cat = (fp64 ? e->prep.has_cat : e->bprep.has_cat) ? 1 : 0;
    a.phi = phi;
    a.status = e->d_status;
    a.q = q;
    a.qd = qd;
    const int64_t chunks = (b.n_paths + a.paths_per_block - 1) / a.paths_per_block;
    const int64_t blocks = chunks * a.n_tiles;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const size_t smem = fwd_smem_bytes(F, a.sub, b.D, fp64, a.ntiles, a.gphi != 0, a.nphi);
    if (smem > kSmemMax) return cudaErrorInvalidConfiguration;
    // nodes per register pass: the tuned count, halved until it divides the rule's
    // padded node count (every smaller power of two then divides it too)
    int np = std::max(2, tn.np);
    while (np > 2 && q.n_pad % np != 0) np /= 2;
    if (!fp64 && q.n_pad % 2 != 0) return cudaErrorInvalidValue;
    switch (b.D) {
#define QTS_CASE(DD) \
    case DD: return launch_fwd_d<DD>(a, np, fp64, warps, blocks, smem, st);
        QTS_CASE(1) QTS_CASE(2) QTS_CASE(3) QTS_CASE(4) QTS_CASE(5) QTS_CASE(6) QTS_CASE(7)
        QTS_CASE(8) QTS_CASE(9) QTS_CASE(10) QTS_CASE(11) QTS_CASE(12) QTS_CASE(13) QTS_CASE(14)
        QTS_CASE(15) QTS_CASE(16) QTS_CASE(20) QTS_CASE(24) QTS_CASE(28) QTS_CASE(32)
        QTS_CASE(40) QTS_CASE(48) QTS_CASE(56) QTS_CASE(64)
#undef QTS_CASE
        default: return cudaErrorInvalidValue;
    }
}


}  // namespace qts

#endif  // QTS_HOST_PART
