// Batched forward + adjoint of many heterogeneous requests in one persistent
// kernel, captured (with its initialisation and epilogues) into a CUDA graph.
//
// Work items are (request, bucket, path chunk, sample tile of 32).  Items are
// not materialised: segments (request, bucket) are ordered by per-item cost,
// heaviest first, and carry their first item index, so a block that takes
// item k from the atomic counter finds its segment by binary search.  For a
// request with grad_phi one pass over each (sample, path) yields both phi and
// the adjoint sums (the forward products P_j S_j are part of the adjoint's).
//
// qts-build-parts: 9 (part 0: host code; parts 1-8: one register class each)
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>

#include "qts_paths.cuh"

namespace qts {

struct SegDev {
    const Rec32* rec;
    double* g_val;      // bucket-offset adjoint accumulators (nullptr: forward only)
    double* g_slot;
    int64_t n_paths;
    int64_t item_begin;
    int32_t D;
    int32_t paths;      // paths per item
    int32_t n_tiles;    // sample groups per chunk (a group = 32, or 32 per warp when priv)
    int32_t req;
    int32_t priv;       // 0: warps share 32 samples (atomics); 1: each warp owns 32
                        // samples and a private phi tile; 2: each warp owns 64
                        // samples, two per lane (sample-pair packing), private tile;
                        // 3: as 2, but the warps share 64 samples and split the paths
    int32_t pad;
};

// Widths that run the fused pass with sample-pair packing when the 64-sample
// tile fits the class's shared memory.  The register classes below are cut so
// that every packed width fits its class's cap without spilling.
__host__ __device__ constexpr bool pair_width(int D) { return D <= 16; }
constexpr int kBatchWarps = 4;

// Per request: x and grad_phi transposed to [feature][Mpad] (row F of XT is
// zero for padding elements; columns >= M are zero), so a warp reads one
// feature of its 32 samples as one coalesced 128-byte line.
struct ReqDev {
    const float* XT;
    const float* GT;    // nullptr: forward only
    double* phi;
    int64_t M;
    int64_t Mpad;
    int32_t F;
    int32_t pad;
    const int* has_nan;
    int* status;
};

struct BatchArgs {
    const SegDev* segs;
    int n_segs;
    const ReqDev* reqs;
    int64_t n_items;
    unsigned long long* counter;
    int64_t tile_floats;  // floats of the phi region (max over the launch's requests)
    int sub;
    QuadF q;
};

// samples per item for each mode
__host__ __device__ __forceinline__ int item_samples(int priv) {
    return priv == 3 ? 64 : priv == 2 ? 64 * kBatchWarps : (priv == 1 ? 32 * kBatchWarps : 32);
}

// floats of the phi region a request needs in a mode
inline int64_t tile_floats_for(int priv, int F) {
    return priv >= 2 ? (int64_t)kBatchWarps * (F + 1) * kTileLd2
                     : (priv == 1 ? (int64_t)kBatchWarps * (F + 1) * kTileLd : (int64_t)(F + 1) * kTileLd);
}

inline size_t batch_smem_bytes(int64_t tile_floats, int sub, int dmax) {
    size_t off = (size_t)tile_floats * 4;
    off = (off + 15) & ~(size_t)15;
    off += 2 * (size_t)sub * (dmax + 1) * sizeof(Rec32);
    off = (off + 15) & ~(size_t)15;
    return off + 16;
}

// node-group width and register policy per width (fits 3 blocks of 128 threads)
template <int D>
struct BatchNP {
    static constexpr bool packed = D <= 16;  // bwd_path_f32_pk
    static constexpr int fused = 2;          // otherwise: lean per-pass variant
    static constexpr bool recomp = true;
    static constexpr int fwd = D <= 8 ? 8 : 2;
};

template <int C>
cudaError_t launch_batch_class(const BatchArgs& a, size_t smem, cudaStream_t st, int* blocks_out, int occ = 0);

#if QTS_DEVICE_PARTS

template <int D>
__device__ __forceinline__ bool batch_item(const SegDev& sg, const ReqDev& rq, int64_t p0, int64_t p1,
                                           int64_t s0, float* ps, Rec32* st0, Rec32* st1, uint64_t* bars,
                                           uint32_t* s_phase, int* s_flag, int sub, const QuadF& q,
                                           float2* zs_all) {
    const int F = rq.F;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (pair_width(D)) {
        if (sg.priv >= 2) {
            // sample-pair modes, lane l the pair 2l, 2l+1 of its warp's 64 samples.
            // priv 2: warp w owns samples s0 + 64 w .. + 63 and walks every path;
            // priv 3: the block's warps share samples s0 .. s0 + 63 and split the
            // paths.  Either way warp w accumulates into its own phi tile w.
            const bool split = sg.priv == 2;
            const int tile_elems = (F + 1) * kTileLd2;
            float* my = ps + warp * tile_elems;
            float2* zs = zs_all + warp * 16;
            const int64_t sw = split ? s0 + 64 * warp : s0;
            for (int idx = lane; idx < tile_elems; idx += 32) my[idx] = 0.f;
            __syncthreads();
            const bool has_nan = *rq.has_nan != 0;
            const GlobalCols2 xr{rq.XT, rq.Mpad, sw + 2 * lane};
            const GlobalCols2 gr{rq.GT, rq.Mpad, sw + 2 * lane};
            const bool ok = stream_paths<Rec32, D>(
                sg.rec, p0, p1, sub, st0, st1, bars, s_phase, s_flag, rq.status,
                [&](int64_t p, const Rec32* r) {
                    double* gsl = sg.g_slot + p * D;
                    double* gv = sg.g_val + 2 * p;
                    if (has_nan) bwd_path_f32_sp<D, true, true>(r, xr, gr, my, zs, lane, q, gsl, gv);
                    else bwd_path_f32_sp<D, false, true>(r, xr, gr, my, zs, lane, q, gsl, gv);
                },
                split);
            if (!ok) return false;
            if (rq.phi) {
                if (split) {
                    for (int idx = lane; idx < 64 * F; idx += 32) {
                        const int s = idx / F, f = idx - s * F;
                        if (sw + s < rq.M) {
                            const float v = my[f * kTileLd2 + s];
                            if (v != 0.f) atomicAdd(&rq.phi[(sw + s) * (F + 1) + f], (double)v);
                        }
                    }
                } else {
                    // stream_paths ended on a block barrier: every warp's tile is complete
                    for (int idx = threadIdx.x; idx < 64 * F; idx += blockDim.x) {
                        const int s = idx / F, f = idx - s * F;
                        if (sw + s < rq.M) {
                            float v = 0.f;
#pragma unroll
                            for (int w = 0; w < kBatchWarps; ++w) v += ps[w * tile_elems + f * kTileLd2 + s];
                            if (v != 0.f) atomicAdd(&rq.phi[(sw + s) * (F + 1) + f], (double)v);
                        }
                    }
                }
            }
            __syncthreads();
            return true;
        }
    }
    const bool priv = sg.priv != 0;
    const int tile_elems = (F + 1) * kTileLd;
    // private mode: warp w owns samples s0 + 32 w .. and tile w
    float* my = priv ? ps + warp * tile_elems : ps;
    const int64_t sw = priv ? s0 + 32 * warp : s0;
    if (priv) {
        for (int idx = lane; idx < tile_elems; idx += 32) my[idx] = 0.f;
    } else {
        for (int idx = threadIdx.x; idx < tile_elems; idx += blockDim.x) ps[idx] = 0.f;
    }
    __syncthreads();
    const bool has_nan = *rq.has_nan != 0;
    const bool grad = rq.GT != nullptr;
    const GlobalCols xr{rq.XT, rq.Mpad, sw + lane};
    const GlobalCols gr{rq.GT, rq.Mpad, sw + lane};
    constexpr int FWD_NP = BatchNP<D>::fwd;
    const bool ok = stream_paths<Rec32, D>(
        sg.rec, p0, p1, sub, st0, st1, bars, s_phase, s_flag, rq.status,
        [&](int64_t p, const Rec32* r) {
            if (grad) {
                double* gsl = sg.g_slot + p * D;
                double* gv = sg.g_val + 2 * p;
                if (priv) {
                    if (has_nan) bwd_path_f32_pk<D, true, kPhiPrivate, GlobalCols, GlobalCols, true>(r, xr, gr, my, lane, q, gsl, gv);
                    else bwd_path_f32_pk<D, false, kPhiPrivate, GlobalCols, GlobalCols, true>(r, xr, gr, my, lane, q, gsl, gv);
                } else {
                    if (has_nan) bwd_path_f32_pk<D, true, kPhiAtomic, GlobalCols, GlobalCols, true>(r, xr, gr, my, lane, q, gsl, gv);
                    else bwd_path_f32_pk<D, false, kPhiAtomic, GlobalCols, GlobalCols, true>(r, xr, gr, my, lane, q, gsl, gv);
                }
            } else {
                auto fwd = [&](auto np) {
                    constexpr int NP = decltype(np)::value;
                    if (priv) {
                        if (has_nan) fwd_path_f32<D, NP, true, GlobalCols, kPhiPrivate, true>(r, xr, my, lane, q);
                        else fwd_path_f32<D, NP, false, GlobalCols, kPhiPrivate, true>(r, xr, my, lane, q);
                    } else {
                        if (has_nan) fwd_path_f32<D, NP, true, GlobalCols, kPhiAtomic, true>(r, xr, my, lane, q);
                        else fwd_path_f32<D, NP, false, GlobalCols, kPhiAtomic, true>(r, xr, my, lane, q);
                    }
                };
                // a rule of fewer than FWD_NP points (or not a multiple of it)
                // runs node pairs
                if (FWD_NP > 2 && q.n_pad % FWD_NP != 0) fwd(std::integral_constant<int, 2>{});
                else fwd(std::integral_constant<int, FWD_NP>{});
            }
        },
        priv);
    if (!ok) return false;
    if (rq.phi) {
        if (priv) {
            for (int idx = lane; idx < 32 * F; idx += 32) {
                const int s = idx / F, f = idx - s * F;
                if (sw + s < rq.M) {
                    const float v = my[f * kTileLd + s];
                    if (v != 0.f) atomicAdd(&rq.phi[(sw + s) * (F + 1) + f], (double)v);
                }
            }
        } else {
            for (int idx = threadIdx.x; idx < 32 * F; idx += blockDim.x) {
                const int s = idx / F, f = idx - s * F;
                if (s0 + s < rq.M) {
                    const float v = ps[f * kTileLd + s];
                    if (v != 0.f) atomicAdd(&rq.phi[(s0 + s) * (F + 1) + f], (double)v);
                }
            }
        }
    }
    __syncthreads();  // the tiles are rewritten by the next item
    return true;
}

// Register classes: DCLASS 8 handles widths 1..6 (4 blocks of 128 threads per
// SM, 128 registers), 12 handles 7..10 (3 blocks, 168 registers), 16 handles
// 11..16 (2 blocks, 255 registers), 32 handles 20..32, and each of the widths
// 40, 48, 56 and 64 (which spill) is a class of its own.
// With two samples per lane a width needs about as many registers as twice
// that width with one, so the cuts sit lower than the widths' names suggest.
template <int DCLASS>
__global__ void __launch_bounds__(128, DCLASS == 8 ? 4 : (DCLASS == 12 ? 3 : (DCLASS == 16 ? 2 : 1)))
    batch_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* ps = (float*)smem;
    size_t off = ((size_t)a.tile_floats * 4 + 15) & ~(size_t)15;
    Rec32* st0 = (Rec32*)(smem + off);
    Rec32* st1 = st0 + (size_t)a.sub * (DCLASS + 1);
    uint64_t* bars = (uint64_t*)(st1 + (size_t)a.sub * (DCLASS + 1));
    __shared__ int s_flag;
    __shared__ uint32_t s_phase[2];
    __shared__ long long s_item;
    __shared__ float2 s_zs[kBatchWarps * 16];
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
        s_phase[0] = s_phase[1] = 0;
    }
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.counter, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        __syncthreads();
        if (item >= a.n_items) break;
        int lo = 0, hi = a.n_segs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.segs[mid].item_begin <= item) lo = mid;
            else hi = mid - 1;
        }
        const SegDev sg = a.segs[lo];
        const ReqDev rq = a.reqs[sg.req];
        const int64_t local = item - sg.item_begin;
        const int64_t s0 = (local % sg.n_tiles) * item_samples(sg.priv);
        const int64_t p0 = (local / sg.n_tiles) * sg.paths;
        const int64_t p1 = imin64(p0 + sg.paths, sg.n_paths);
        bool ok = true;
#define QTS_CASE(DD) \
    case DD: ok = batch_item<DD>(sg, rq, p0, p1, s0, ps, st0, st1, bars, s_phase, &s_flag, a.sub, a.q, s_zs); break;
        if constexpr (DCLASS == 8) {
            switch (sg.D) {
                QTS_CASE(1) QTS_CASE(2) QTS_CASE(3) QTS_CASE(4) QTS_CASE(5) QTS_CASE(6)
                default: break;
            }
        } else if constexpr (DCLASS == 12) {
            switch (sg.D) {
                QTS_CASE(7) QTS_CASE(8) QTS_CASE(9) QTS_CASE(10)
                default: break;
            }
        } else if constexpr (DCLASS == 16) {
            switch (sg.D) {
                QTS_CASE(11) QTS_CASE(12) QTS_CASE(13) QTS_CASE(14) QTS_CASE(15) QTS_CASE(16)
                default: break;
            }
        } else if constexpr (DCLASS == 32) {
            switch (sg.D) {
                QTS_CASE(20) QTS_CASE(24) QTS_CASE(28) QTS_CASE(32)
                default: break;
            }
        } else {
            switch (sg.D) {
                QTS_CASE(DCLASS)
                default: break;
            }
        }
#undef QTS_CASE
        if (!ok) break;  // a bounded wait ran out: status is set, stop this block
    }
}

// occ > 0: at most occ blocks per SM (the persistent grid is occ x SMs blocks)
template <int C>
cudaError_t launch_batch_class(const BatchArgs& a, size_t smem, cudaStream_t st, int* blocks_out, int occ) {
    auto k = batch_kernel<C>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, smem);
    if (e != cudaSuccess) return e;
    if (occ > 0) per_sm = std::min(per_sm, occ);
    const int blocks = std::max(1, per_sm) * num_sms();
    *blocks_out = blocks;
    k<<<blocks, 128, smem, st>>>(a);
    return cudaGetLastError();
}

#define QTS_INST(C) \
    template cudaError_t launch_batch_class<C>(const BatchArgs&, size_t, cudaStream_t, int*, int);
#if QTS_IN_PART(1)
QTS_INST(8)
#endif
#if QTS_IN_PART(2)
QTS_INST(12)
#endif
#if QTS_IN_PART(3)
QTS_INST(16)
#endif
#if QTS_IN_PART(4)
QTS_INST(32)
#endif
#if QTS_IN_PART(5)
QTS_INST(40)
#endif
#if QTS_IN_PART(6)
QTS_INST(48)
#endif
#if QTS_IN_PART(7)
QTS_INST(56)
#endif
#if QTS_IN_PART(8)
QTS_INST(64)
#endif
#undef QTS_INST

#endif  // QTS_DEVICE_PARTS

#if !QTS_HOST_PART
}  // namespace qts
#endif

#if QTS_HOST_PART

// out[c * Mpad + s] = in[s * ld + c] for c < ncols, s < M; zero elsewhere
// (rows up to nrows, columns up to Mpad).
__global__ void transpose_pad_kernel(const float* __restrict__ in, int64_t M, int ncols, int64_t ld,
                                     float* __restrict__ out, int nrows, int64_t Mpad, int* has_nan) {
    __shared__ float tile[32][33];
    const int64_t s0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    int nan_seen = 0;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t s = s0 + r;
        const int c = c0 + threadIdx.x;
        float v = 0.f;
        if (s < M && c < ncols) v = in[s * ld + c];
        nan_seen |= (v != v);
        tile[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r;
        const int64_t s = s0 + threadIdx.x;
        if (c < nrows && s < Mpad) out[(int64_t)c * Mpad + s] = tile[threadIdx.x][r];
    }
    if (has_nan && nan_seen) atomicOr(has_nan, 1);
}

// ------------------------------------------------------------- host side --

struct BatchPlan {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    void* dev = nullptr;  // segments, requests, counters
    int kernels = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the persistent kernel(s)
};

static std::mutex g_plan_mu;
static std::vector<BatchPlan*> g_plans;  // most recent last
static thread_local BatchPlan* g_last_plan = nullptr;
// cached graphs (a caller that launches each of many requests on its own keeps
// one plan per request)
constexpr size_t kMaxPlans = 256;

static void destroy_plan(BatchPlan* p) {
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->dev) cudaFree(p->dev);
    delete p;
}

// drop every cached plan that mentions this ensemble (called before it is freed
// or its device memory moves)
void batch_forget(const qts_ensemble* e) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    const uint64_t id = (uint64_t)(uintptr_t)e;
    for (size_t i = 0; i < g_plans.size();) {
        const auto& k = g_plans[i]->key;
        if (std::find(k.begin(), k.end(), id) != k.end()) {
            cudaDeviceSynchronize();
            if (g_last_plan == g_plans[i]) g_last_plan = nullptr;
            destroy_plan(g_plans[i]);
            g_plans.erase(g_plans.begin() + i);
        } else {
            ++i;
        }
    }
}

// widths 40, 48, 56 and 64 (bucket widths) are classes of their own
int batch_class(int D) { return D <= 6 ? 8 : D <= 10 ? 12 : (D <= 16 ? 16 : (D <= 32 ? 32 : D)); }
// shared memory one block of a class may use and still reach its blocks per SM
static size_t class_smem_budget(int cls) {
    const size_t sm = 227 * 1024;
    const int blocks = cls == 8 ? 4 : cls == 12 ? 3 : cls == 16 ? 2 : 1;
    return sm / blocks - 1024;
}

// paths per work item: about 2^23 FP32 operations per item
static int item_paths(int D, bool grad) {
    const int per_path = 32 * 8 * D * (grad ? 12 : 4);
    int p = (1 << 23) / std::max(per_path, 1);
    p = std::max(32, std::min(2048, p));
    return (p + 31) / 32 * 32;
}

cudaError_t launch_bwd_epilogue(const qts_ensemble* e, const float* grad, int64_t M, int F,
                                const double* g_val, const double* g_slot, double* d_leaf,
                                double* d_z, double* gb, cudaStream_t st);

// Workspace of one request in its ensemble: [adjoint sums (grad only)][XT][GT (grad only)][flag]
struct BatchWork {
    size_t grad_bytes, xt_off, gt_off, flag_off, total;
    int64_t Mpad;
};

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

static BatchWork batch_work(const qts_ensemble* e, int64_t M, int F, bool grad) {
    BatchWork w;
    w.Mpad = (M + 64 * kBatchWarps - 1) / (64 * kBatchWarps) * (64 * kBatchWarps);
    // adjoint sums of the pair tables: two per path (a sibling pair's two leaves), one per slot
    w.grad_bytes = grad ? align256(sizeof(double) * (size_t)(4 + 2 * e->bprep.n_paths + e->bprep.n_slots)) : 0;
    const size_t tbytes = align256(sizeof(float) * (size_t)(F + 1) * (size_t)w.Mpad);
    w.xt_off = w.grad_bytes;
    w.gt_off = w.xt_off + tbytes;
    w.flag_off = w.gt_off + (grad ? tbytes : 0);
    w.total = w.flag_off + 256;
    return w;
}

static cudaError_t launch_transpose(const float* in, int64_t M, int ncols, int64_t ld, float* out, int nrows,
                                    int64_t Mpad, int* has_nan, cudaStream_t st) {
    if (Mpad == 0) return cudaSuccess;
    dim3 grid((unsigned)(Mpad / 32), (unsigned)((nrows + 31) / 32));
    transpose_pad_kernel<<<grid, dim3(32, 8), 0, st>>>(in, M, ncols, ld, out, nrows, Mpad, has_nan);
    return cudaGetLastError();
}

// Requests with F + 1 <= kPrivRows use per-warp private phi tiles (plain
// read-add-write); wider ones share one tile with shared-memory atomics.
constexpr int kPrivRows = 64;

// Per-width launch choices that override the ensembles' own while tuning:
// paths per work item and packed sample mapping (0: keep), and optionally only
// the buckets of one width.
struct BatchOverride {
    int paths[kMaxD + 1];
    int mode[kMaxD + 1];
    int occ[kMaxD + 1];  // blocks per SM of the width's class (0: the tuned or full count)
    int only_width;
    int only_class;      // > 0: only the widths of this register class
};

static qts_status build_plan(int n, const qts_request* reqs, int n_quad, BatchPlan* plan,
                             cudaStream_t cap, const BatchOverride* ov = nullptr) {
    struct SegHost {
        SegDev d;
        double cost;  // per item
        int cls;
        int64_t tile;  // floats of its phi region
        int bin;       // tile-size bin: one launch per (class, bin, rule)
        int occ;       // blocks per SM of its class launch (0: as many as fit)
        int nq;        // quadrature points of the bucket (QTS_NQ_EXACT: ceil(D/2))
        int npad;      // ... padded to what its variant of the pass takes per register pass
    };
    std::vector<SegHost> segs;
    std::vector<ReqDev> rd(n);
    const int sub = 32;                        // paths per staged sub-chunk
    for (int r = 0; r < n; ++r) {
        const qts_request& R = reqs[r];
        qts_ensemble* e = R.ens;
        const bool grad = R.grad_phi != nullptr;
        const BatchWork bw = batch_work(e, R.M, R.F, grad);
        char* wbase = (char*)e->d_work;
        rd[r] = {(const float*)(wbase + bw.xt_off), grad ? (const float*)(wbase + bw.gt_off) : nullptr, R.phi,
                 R.M, bw.Mpad, R.F, 0, (const int*)(wbase + bw.flag_off), e->d_status};
        if (R.M <= 0) continue;
        double* g_val = grad ? (double*)e->d_work + 4 : nullptr;
        double* g_slot = grad ? g_val + 2 * e->bprep.n_paths : nullptr;
        for (const Bucket& b : e->bprep.buckets) {
            if (ov && ov->only_width > 0 && b.D != ov->only_width) continue;
            const int cls = batch_class(b.D);
            if (ov && ov->only_class > 0 && cls != ov->only_class) continue;
            const Tune& tn = e->tune[b.D];
            int mode = R.F + 1 <= kPrivRows ? 1 : 0;
            if (grad && pair_width(b.D) &&
                batch_smem_bytes(tile_floats_for(2, R.F), sub, cls) <= class_smem_budget(cls)) {
                const int want = ov && ov->mode[b.D] ? ov->mode[b.D] : tn.bt_mode;
                mode = want == 3 ? 3 : 2;
            }
            const int per_item = item_samples(mode);
            const int n_tiles = (int)((R.M + per_item - 1) / per_item);
            SegHost s;
            s.d.rec = (const Rec32*)e->bdev.rec + b.rec_off;
            s.d.g_val = grad ? g_val + 2 * b.path_base : nullptr;
            s.d.g_slot = grad ? g_slot + b.slot_base : nullptr;
            s.d.n_paths = b.n_paths;
            s.d.D = b.D;
            s.d.paths = ov && ov->paths[b.D] ? ov->paths[b.D]
                        : tn.bt_paths ? tn.bt_paths : (e->tuned ? tn.bpaths : item_paths(b.D, grad));
            s.d.n_tiles = n_tiles;
            s.d.req = r;
            s.d.priv = mode;
            s.d.pad = 0;
            s.occ = ov && ov->occ[b.D] ? ov->occ[b.D] : tn.bt_occ;
            s.nq = nodes_for(n_quad, b.D, 1);
            // the packed fused pass takes one node at a time, the others node pairs
            const int pad = (grad && mode >= 2) ? 1 : 2;
            s.npad = (s.nq + pad - 1) / pad * pad;
            s.cost = (double)s.d.paths * b.D * (grad ? 12 : 4) * s.npad;
            s.cls = cls;
            // a launch sizes its shared memory for its widest tile, and whatever
            // shared memory a block does not take stays L1 (which serves the x and
            // grad_phi loads): requests of one class are launched by tile size
            s.tile = tile_floats_for(mode, R.F);
            const int64_t tb = s.tile * 4;
            s.bin = tb <= 48 * 1024 ? 0 : tb <= 80 * 1024 ? 1 : 2;
            segs.push_back(s);
        }
    }
    // one launch per (kernel class, tile bin, quadrature rule), heaviest items
    // first within it
    std::stable_sort(segs.begin(), segs.end(), [](const SegHost& a, const SegHost& b) {
        if (a.cls != b.cls) return a.cls < b.cls;
        if (a.bin != b.bin) return a.bin < b.bin;
        if (a.npad != b.npad) return a.npad > b.npad;
        if (a.nq != b.nq) return a.nq > b.nq;
        return a.cost > b.cost;
    });
    std::vector<int> cls_list, cls_nq, cls_npad, cls_occ;
    std::vector<int64_t> cls_items, cls_first_seg, cls_tile;
    int64_t item = 0;
    for (size_t i = 0; i < segs.size(); ++i) {
        if (cls_list.empty() || cls_list.back() != segs[i].cls || segs[i - 1].bin != segs[i].bin ||
            segs[i - 1].nq != segs[i].nq || segs[i - 1].npad != segs[i].npad) {
            cls_list.push_back(segs[i].cls);
            cls_nq.push_back(segs[i].nq);
            cls_npad.push_back(segs[i].npad);
            cls_occ.push_back(0);
            cls_first_seg.push_back((int64_t)i);
            cls_items.push_back(0);
            cls_tile.push_back(0);
            item = 0;
        }
        cls_tile.back() = std::max(cls_tile.back(), segs[i].tile);
        // a launch takes the smallest cap of its widths
        if (segs[i].occ > 0 && (cls_occ.back() == 0 || segs[i].occ < cls_occ.back())) cls_occ.back() = segs[i].occ;
        segs[i].d.item_begin = item;
        const int64_t chunks = (segs[i].d.n_paths + segs[i].d.paths - 1) / segs[i].d.paths;
        item += chunks * segs[i].d.n_tiles;
        cls_items.back() = item;
    }
    const size_t seg_bytes = (sizeof(SegDev) * std::max<size_t>(segs.size(), 1) + 255) / 256 * 256;
    const size_t req_bytes = (sizeof(ReqDev) * std::max(n, 1) + 255) / 256 * 256;
    const size_t cnt_bytes = 256;
    cudaError_t ce = cudaMalloc(&plan->dev, seg_bytes + req_bytes + cnt_bytes);
    if (ce != cudaSuccess) return cuda_fail(ce, "batch plan allocation");
    SegDev* d_segs = (SegDev*)plan->dev;
    ReqDev* d_reqs = (ReqDev*)((char*)plan->dev + seg_bytes);
    unsigned long long* d_cnt = (unsigned long long*)((char*)plan->dev + seg_bytes + req_bytes);
    std::vector<SegDev> sd(segs.size());
    for (size_t i = 0; i < segs.size(); ++i) sd[i] = segs[i].d;
    if (!sd.empty()) ce = cudaMemcpy(d_segs, sd.data(), sizeof(SegDev) * sd.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(d_reqs, rd.data(), sizeof(ReqDev) * n, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return cuda_fail(ce, "batch plan upload");

    ce = cudaEventCreate(&plan->ev0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&plan->ev1);
    if (ce != cudaSuccess) return cuda_fail(ce, "batch plan events");
    // capture: init, persistent kernel(s), epilogues
    ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph capture begin");
    int kernels = 0;
    cudaError_t err = cudaSuccess;
    for (int r = 0; r < n && err == cudaSuccess; ++r) {
        const qts_request& R = reqs[r];
        const bool grad = R.grad_phi != nullptr;
        const BatchWork bw = batch_work(R.ens, R.M, R.F, grad);
        char* wbase = (char*)R.ens->d_work;
        if (R.phi && R.M > 0) {
            err = launch_phi_init(R.phi, R.M, R.F, R.ens->bprep.bias, cap);
            ++kernels;
        }
        if (grad && err == cudaSuccess) err = cudaMemsetAsync(wbase, 0, bw.grad_bytes, cap);
        // the NaN flag starts set for ensembles with categorical elements, so
        // their items take the NaN-aware (categorical-aware) variant
        if (err == cudaSuccess)
            err = cudaMemsetAsync(wbase + bw.flag_off, R.ens->bprep.has_cat ? 1 : 0, 256, cap);
        if (R.M > 0 && err == cudaSuccess) {
            err = launch_transpose(R.X, R.M, R.F, R.F, (float*)(wbase + bw.xt_off), R.F + 1, bw.Mpad,
                                   (int*)(wbase + bw.flag_off), cap);
            ++kernels;
            if (grad && err == cudaSuccess) {
                err = launch_transpose(R.grad_phi, R.M, R.F + 1, R.F + 1, (float*)(wbase + bw.gt_off), R.F + 1,
                                       bw.Mpad, nullptr, cap);
                ++kernels;
            }
        }
    }
    if (err == cudaSuccess) err = cudaMemsetAsync(d_cnt, 0, cnt_bytes, cap);
    if (err == cudaSuccess) err = cudaEventRecordWithFlags(plan->ev0, cap, cudaEventRecordExternal);
    for (size_t c = 0; c < cls_list.size() && err == cudaSuccess; ++c) {
        const int cls = cls_list[c];
        BatchArgs a;
        a.segs = d_segs + cls_first_seg[c];
        a.n_segs = (int)((c + 1 < cls_list.size() ? cls_first_seg[c + 1] : (int64_t)segs.size()) - cls_first_seg[c]);
        a.reqs = d_reqs;
        a.n_items = cls_items[c];
        a.counter = d_cnt + c;
        a.tile_floats = std::max<int64_t>(cls_tile[c], kTileLd);
        a.sub = sub;
        if (!make_quad(cls_nq[c], &a.q, nullptr, cls_npad[c] == cls_nq[c] ? 1 : 2) || a.q.n_pad != cls_npad[c]) {
            err = cudaErrorInvalidValue;
            break;
        }
        const size_t smem = batch_smem_bytes(a.tile_floats, sub, cls);
        int blocks = 0;
        if (cls == 8) err = launch_batch_class<8>(a, smem, cap, &blocks, cls_occ[c]);
        else if (cls == 12) err = launch_batch_class<12>(a, smem, cap, &blocks, cls_occ[c]);
        else if (cls == 16) err = launch_batch_class<16>(a, smem, cap, &blocks, cls_occ[c]);
        else if (cls == 32) err = launch_batch_class<32>(a, smem, cap, &blocks, cls_occ[c]);
        else if (cls == 40) err = launch_batch_class<40>(a, smem, cap, &blocks, cls_occ[c]);
        else if (cls == 48) err = launch_batch_class<48>(a, smem, cap, &blocks, cls_occ[c]);
        else if (cls == 56) err = launch_batch_class<56>(a, smem, cap, &blocks, cls_occ[c]);
        else err = launch_batch_class<64>(a, smem, cap, &blocks, cls_occ[c]);
        ++kernels;
    }
    if (err == cudaSuccess) err = cudaEventRecordWithFlags(plan->ev1, cap, cudaEventRecordExternal);
    for (int r = 0; r < n && err == cudaSuccess; ++r) {
        const qts_request& R = reqs[r];
        if (!R.grad_phi) continue;
        double* gb = (double*)R.ens->d_work;
        double* g_val = gb + 4;
        double* g_slot = g_val + 2 * R.ens->bprep.n_paths;
        if (R.M > 0) {
            err = launch_bwd_epilogue_pairs(R.ens, R.grad_phi, R.M, R.F, g_val, g_slot, R.d_leaf, R.d_z, gb, cap);
            kernels += 1 + (R.ens->bprep.n_paths + (int64_t)R.ens->bprep.empty_leaf.size() > 0) +
                       (R.ens->bprep.n_slots > 0);
        } else {
            err = cudaMemsetAsync(R.d_leaf, 0, sizeof(double) * R.ens->n_nodes, cap);
            if (err == cudaSuccess) err = cudaMemsetAsync(R.d_z, 0, sizeof(double) * R.ens->n_nodes, cap);
        }
    }
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(cap, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(err, "batched launch during capture");
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "graph capture end");
    plan->graph = g;
    ce = cudaGraphInstantiate(&plan->exec, g, 0);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiate");
    plan->kernels = kernels;
    return QTS_OK;
}

static thread_local int g_last_batch_kernels = 0;

}  // namespace qts

using namespace qts;

namespace qts {

// Argument checks shared by the batched call and its tuner; grows every
// request's workspace to what the batched launch needs.
static qts_status check_batch(int32_t n, const qts_request* reqs, int32_t n_quad) {
    if (n < 1 || !reqs) return fail(QTS_ERR_ARG, "no requests");
    for (int r = 0; r < n; ++r) {
        const qts_request& R = reqs[r];
        qts_status st = check_call(R.ens, R.X, R.M, R.F, n_quad);
        if (st != QTS_OK) return fail(st, "request " + std::to_string(r) + ": " + qts_last_error());
        if (R.ens->flags & QTS_FLAG_FP64)
            return fail(QTS_ERR_UNSUPPORTED, "request " + std::to_string(r) + ": batched calls use FP32 tables");
        if (!R.grad_phi && !R.phi) return fail(QTS_ERR_ARG, "request " + std::to_string(r) + ": nothing to compute");
        if (R.grad_phi && (!R.d_leaf || !R.d_z))
            return fail(QTS_ERR_ARG, "request " + std::to_string(r) + ": d_leaf/d_z are NULL");
        for (int s = 0; s < r; ++s)
            if (reqs[s].ens == R.ens)
                return fail(QTS_ERR_ARG, "an ensemble may appear in at most one request of a batch");
    }
    for (int r = 0; r < n; ++r) {
        const qts_request& R = reqs[r];
        qts_status st = ensure_batch_tables(R.ens);
        if (st != QTS_OK) return st;
        st = ensure_workspace(R.ens, batch_work(R.ens, R.M, R.F, R.grad_phi != nullptr).total);
        if (st != QTS_OK) return st;
    }
    return QTS_OK;
}

}  // namespace qts

extern "C" qts_status qts_batched_fwd_bwd(int32_t n, const qts_request* reqs, int32_t n_quad,
                                          qts_stream_t stream) {
    {
        const qts_status st = check_batch(n, reqs, n_quad);
        if (st != QTS_OK) return st;
    }
    std::vector<uint64_t> key;
    key.push_back((uint64_t)n_quad);
    for (int r = 0; r < n; ++r) {
        const qts_request& R = reqs[r];
        for (uint64_t v : {(uint64_t)(uintptr_t)R.ens, (uint64_t)(uintptr_t)R.X, (uint64_t)R.M, (uint64_t)R.F,
                           (uint64_t)(uintptr_t)R.grad_phi, (uint64_t)(uintptr_t)R.phi,
                           (uint64_t)(uintptr_t)R.d_leaf, (uint64_t)(uintptr_t)R.d_z,
                           (uint64_t)(uintptr_t)R.ens->d_work, (uint64_t)(uintptr_t)R.ens->bdev.rec,
                           (uint64_t)R.ens->tune_gen})
            key.push_back(v);
    }
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (size_t i = 0; i < g_plans.size(); ++i) {
            if (g_plans[i]->key == key) {
                BatchPlan* p = g_plans[i];
                g_plans.erase(g_plans.begin() + i);
                g_plans.push_back(p);
                exec = p->exec;
                g_last_batch_kernels = p->kernels;
                g_last_plan = p;
                break;
            }
        }
    }
    if (!exec) {
        cudaStream_t cap;
        cudaError_t ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (ce != cudaSuccess) return cuda_fail(ce, "capture stream");
        auto* plan = new BatchPlan();
        plan->key = key;
        qts_status st = build_plan(n, reqs, n_quad, plan, cap);
        cudaStreamDestroy(cap);
        if (st != QTS_OK) {
            destroy_plan(plan);
            return st;
        }
        std::lock_guard<std::mutex> lk(g_plan_mu);
        if (g_plans.size() >= kMaxPlans) {
            cudaDeviceSynchronize();
            if (g_last_plan == g_plans.front()) g_last_plan = nullptr;
            destroy_plan(g_plans.front());
            g_plans.erase(g_plans.begin());
        }
        g_plans.push_back(plan);
        exec = plan->exec;
        g_last_batch_kernels = plan->kernels;
        g_last_plan = plan;
    }
    cudaError_t ce = cudaGraphLaunch(exec, (cudaStream_t)stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph launch");
    return QTS_OK;
}

namespace qts {

// Device time of the persistent kernels of one plan built for `reqs` with the
// override `ov` (second of two launches); the plan is destroyed afterwards.
static qts_status time_plan(int n, const qts_request* reqs, int n_quad, const BatchOverride& ov,
                            cudaStream_t cap, cudaStream_t st, float* ms) {
    auto* plan = new BatchPlan();
    qts_status s = build_plan(n, reqs, n_quad, plan, cap, &ov);
    cudaError_t ce = cudaSuccess;
    for (int k = 0; k < 2 && s == QTS_OK && ce == cudaSuccess; ++k) ce = cudaGraphLaunch(plan->exec, st);
    if (s == QTS_OK && ce == cudaSuccess) ce = cudaEventSynchronize(plan->ev1);
    if (s == QTS_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(ms, plan->ev0, plan->ev1);
    if (s == QTS_OK && ce != cudaSuccess) s = cuda_fail(ce, "batched tuning run");
    cudaStreamSynchronize(st);
    destroy_plan(plan);
    return s;
}

}  // namespace qts

extern "C" qts_status qts_batched_autotune(int32_t n, const qts_request* reqs, int32_t n_quad, int64_t max_samples,
                                           int32_t* chosen, qts_stream_t stream) {
    qts_status st = check_batch(n, reqs, n_quad);
    if (st != QTS_OK) return st;
    if (max_samples < 0) return fail(QTS_ERR_ARG, "max_samples must be >= 0");
    std::vector<qts_request> sub(reqs, reqs + n);
    if (max_samples > 0)
        for (auto& R : sub) R.M = std::min<int64_t>(R.M, max_samples);
    // work (element-samples) per bucket width of the reduced batch, and whether
    // the width runs the packed fused pass for some request
    std::vector<double> work(kMaxD + 1, 0.0);
    std::vector<char> packed(kMaxD + 1, 0);
    std::vector<char> fused(kMaxD + 1, 0);
    for (const auto& R : sub) {
        if (R.M <= 0) continue;
        for (const Bucket& b : R.ens->bprep.buckets) {
            if (b.n_paths == 0) continue;
            work[b.D] += (double)R.M * (double)b.n_paths * b.D;
            if (R.grad_phi) fused[b.D] = 1;
            if (R.grad_phi && pair_width(b.D)) packed[b.D] = 1;
        }
    }
    double total = 0.0;
    for (double w : work) total += w;
    std::vector<int> widths;
    for (int D = 1; D <= kMaxD; ++D)
        if (work[D] > 0.01 * total) widths.push_back(D);  // the rest keep the defaults
    std::sort(widths.begin(), widths.end(), [&](int a, int b) { return work[a] > work[b]; });
    cudaStream_t cap;
    cudaError_t ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return cuda_fail(ce, "capture stream");
    std::vector<int> best_paths(kMaxD + 1, 0), best_mode(kMaxD + 1, 0);
    for (int D : widths) {
        BatchOverride ov;
        std::memset(&ov, 0, sizeof(ov));
        ov.only_width = D;
        const int base = item_paths(D, fused[D] != 0);
        float best = 1e30f;
        for (int mode : {2, 3}) {
            if (mode == 3 && !packed[D]) continue;
            for (int mult : {1, 2, 4, 8}) {  // base, twice, four and eight times
                const int paths = std::max(32, std::min(4096, base * mult / 32 * 32));
                ov.paths[D] = paths;
                ov.mode[D] = packed[D] ? mode : 0;
                float ms = 0.f;
                st = time_plan(n, sub.data(), n_quad, ov, cap, (cudaStream_t)stream, &ms);
                if (st != QTS_OK) {
                    cudaStreamDestroy(cap);
                    return st;
                }
                if (ms < best) {
                    best = ms;
                    best_paths[D] = paths;
                    best_mode[D] = ov.mode[D];
                }
            }
        }
    }
    // blocks per SM of the two register classes that fit three or more: all
    // that fit, or one fewer, which leaves the SM's shared memory more L1 for
    // the x and grad_phi reads; timed over the class's widths with the choices
    // above
    std::vector<int> best_occ(kMaxD + 1, 0);
    for (int cls : {8, 12}) {
        bool any = false;
        for (int D : widths) any = any || batch_class(D) == cls;
        if (!any) continue;
        const int full = cls == 8 ? 4 : 3;
        BatchOverride ov;
        std::memset(&ov, 0, sizeof(ov));
        ov.only_class = cls;
        for (int D = 1; D <= kMaxD; ++D) {
            ov.paths[D] = best_paths[D];
            ov.mode[D] = best_mode[D];
        }
        float t[2] = {0.f, 0.f};
        for (int k = 0; k < 2; ++k) {
            for (int D = 1; D <= kMaxD; ++D) ov.occ[D] = (k == 1 && batch_class(D) == cls) ? full - 1 : 0;
            st = time_plan(n, sub.data(), n_quad, ov, cap, (cudaStream_t)stream, &t[k]);
            if (st != QTS_OK) {
                cudaStreamDestroy(cap);
                return st;
            }
        }
        if (t[1] < t[0])
            for (int D = 1; D <= kMaxD; ++D)
                if (batch_class(D) == cls) best_occ[D] = full - 1;
    }
    cudaStreamDestroy(cap);
    for (int r = 0; r < n; ++r) {
        qts_ensemble* e = reqs[r].ens;
        for (int D : widths) {
            e->tune[D].bt_paths = best_paths[D];
            e->tune[D].bt_mode = best_mode[D];
        }
        for (int D = 1; D <= kMaxD; ++D) e->tune[D].bt_occ = best_occ[D];
        ++e->tune_gen;
        batch_forget(e);
    }
    if (chosen)
        for (int D = 0; D <= kMaxD; ++D) {
            chosen[3 * D] = best_paths[D];
            chosen[3 * D + 1] = best_mode[D];
            chosen[3 * D + 2] = best_occ[D];
        }
    return QTS_OK;
}

extern "C" qts_status qts_get_batch_info(qts_ensemble* e, int64_t* n_paths, int64_t* sum_unique,
                                         int64_t* n_pair_paths, int32_t* n_buckets, int32_t* bucket_width,
                                         int64_t* bucket_paths) {
    if (!e) return fail(QTS_ERR_ARG, "ensemble handle is NULL");
    if (e->flags & QTS_FLAG_FP64) return fail(QTS_ERR_UNSUPPORTED, "batched calls use FP32 tables");
    const qts_status st = ensure_batch_tables(e);
    if (st != QTS_OK) return st;
    if (n_paths) *n_paths = e->bprep.n_paths;
    if (sum_unique) *sum_unique = e->bprep.sum_unique;
    if (n_pair_paths) *n_pair_paths = e->bprep.n_pair_paths;
    const size_t nb = std::min<size_t>(e->bprep.buckets.size(), 32);
    if (n_buckets) *n_buckets = (int32_t)nb;
    for (size_t i = 0; i < nb; ++i) {
        if (bucket_width) bucket_width[i] = e->bprep.buckets[i].D;
        if (bucket_paths) bucket_paths[i] = e->bprep.buckets[i].n_paths;
    }
    return QTS_OK;
}

extern "C" int32_t qts_batched_kernel_count(void) { return g_last_batch_kernels; }

extern "C" qts_status qts_batched_last_kernel_ms(float* ms) {
    if (!ms) return fail(QTS_ERR_ARG, "ms is NULL");
    std::lock_guard<std::mutex> lk(g_plan_mu);
    if (!g_last_plan || std::find(g_plans.begin(), g_plans.end(), g_last_plan) == g_plans.end())
        return fail(QTS_ERR_ARG, "no batched call on this thread");
    cudaError_t ce = cudaEventSynchronize(g_last_plan->ev1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(ms, g_last_plan->ev0, g_last_plan->ev1);
    return ce == cudaSuccess ? QTS_OK : cuda_fail(ce, "batched kernel timing");
}

#endif  // QTS_HOST_PART
