// C-ABI entry points: handle lifecycle, argument checks, per-bucket launches.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "qts_device.cuh"
#include "qts_internal.h"

namespace qts {

static thread_local std::string g_err = "no error";

void set_error(const std::string& msg) { g_err = msg; }

qts_status fail(qts_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

qts_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? QTS_ERR_OOM : QTS_ERR_CUDA;
}

int num_sms() {
    static int sms = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 152;
    });
    return sms;
}

static Tune default_tune(int D) {
    Tune t;
    t.warps = 4;
    t.sub = D <= 16 ? 32 : 16;
    t.paths = D <= 8 ? 512 : (D <= 16 ? 256 : 128);
    t.np = D <= 8 ? 8 : (D <= 24 ? 4 : 2);
    t.bpaths = 128;
    // forward: up to width 8 the block's warps share a sample tile and split
    // the paths (one phi tile each); wider paths give each warp its own samples
    t.priv = D <= 8 ? 2 : 1;
    return t;
}

void release_device(qts_ensemble* e) {
    cudaFree(e->d_rec);
    cudaFree(e->d_path_leaf);
    cudaFree(e->d_path_zprod);
    cudaFree(e->d_path_val);
    cudaFree(e->d_slot_zexcl);
    cudaFree(e->d_slot_edge_begin);
    cudaFree(e->d_edge_node);
    cudaFree(e->d_edge_coef);
    cudaFree(e->d_empty_leaf);
    e->d_rec = nullptr;
    e->d_path_leaf = nullptr;
    e->d_path_zprod = nullptr;
    e->d_path_val = nullptr;
    e->d_slot_zexcl = nullptr;
    e->d_slot_edge_begin = nullptr;
    e->d_edge_node = nullptr;
    e->d_edge_coef = nullptr;
    e->d_empty_leaf = nullptr;
    e->device_bytes = 0;
    release_dfs(e);
    release_batch_tables(e);
}

void release_batch_tables(qts_ensemble* e) {
    DevTables& T = e->bdev;
    for (void* p : {T.rec, (void*)T.path_leaf, (void*)T.path_zprod, (void*)T.path_val, (void*)T.slot_zexcl,
                    (void*)T.slot_edge_begin, (void*)T.edge_node, (void*)T.edge_coef, (void*)T.empty_leaf,
                    (void*)T.pair_leaf2, (void*)T.pair_zprod2, (void*)T.pair_z, (void*)T.pair_gslot})
        cudaFree(p);
    T = DevTables();
    e->bprep = Prepared();
    e->bready = false;
}

template <typename T>
static qts_status up(T** dst, const std::vector<T>& src, int64_t* total, const char* what) {
    size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    cudaError_t err = cudaMalloc((void**)dst, bytes);
    if (err != cudaSuccess) return cuda_fail(err, what);
    if (!src.empty()) {
        err = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (err != cudaSuccess) return cuda_fail(err, what);
    }
    *total += (int64_t)bytes;
    return QTS_OK;
}

qts_status upload(qts_ensemble* e) {
    const Prepared& P = e->prep;
    int64_t tot = 0;
    qts_status st = QTS_OK;
    if (e->flags & QTS_FLAG_FP64) st = up((Rec64**)&e->d_rec, P.rec64, &tot, "upload path tables");
    else st = up((Rec32**)&e->d_rec, P.rec32, &tot, "upload path tables");
    if (st == QTS_OK) st = up(&e->d_path_leaf, P.path_leaf, &tot, "upload path leaves");
    if (st == QTS_OK) st = up(&e->d_path_zprod, P.path_zprod, &tot, "upload path products");
    if (st == QTS_OK) st = up(&e->d_path_val, P.path_val, &tot, "upload path values");
    if (st == QTS_OK) st = up(&e->d_slot_zexcl, P.slot_zexcl, &tot, "upload element products");
    if (st == QTS_OK) st = up(&e->d_slot_edge_begin, P.slot_edge_begin, &tot, "upload element edges");
    if (st == QTS_OK) st = up(&e->d_edge_node, P.edge_node, &tot, "upload edge nodes");
    if (st == QTS_OK) st = up(&e->d_edge_coef, P.edge_coef, &tot, "upload edge coefficients");
    if (st == QTS_OK) st = up(&e->d_empty_leaf, P.empty_leaf, &tot, "upload single-leaf trees");
    if (st != QTS_OK) {
        release_device(e);
        return st;
    }
    e->device_bytes = tot;
    // the device copies are the working set; keep only sizes and bucket info
    Prepared& Pm = e->prep;
    std::vector<Rec32>().swap(Pm.rec32);
    std::vector<Rec64>().swap(Pm.rec64);
    std::vector<int64_t>().swap(Pm.path_leaf);
    std::vector<double>().swap(Pm.path_zprod);
    std::vector<double>().swap(Pm.path_val);
    std::vector<double>().swap(Pm.slot_zexcl);
    std::vector<int64_t>().swap(Pm.slot_edge_begin);
    std::vector<int64_t>().swap(Pm.edge_node);
    std::vector<double>().swap(Pm.edge_coef);
    return QTS_OK;
}

// Pair tables of the batched pass: prepared from the host copy of the model
// with sibling leaves merged, uploaded, host copies dropped.
qts_status ensure_batch_tables(qts_ensemble* e) {
    if (e->bready) return QTS_OK;
    Prepared& P = e->bprep;
    std::string err;
    const bool cat = !e->is_cat.empty();
    qts_status st = prepare(e->n_trees, e->off.data(), e->left.data(), e->right.data(), e->feature.data(),
                            e->thr.data(), e->defl.data(), e->z.data(), e->leaf.data(),
                            cat ? e->is_cat.data() : nullptr, cat ? e->cat_left.data() : nullptr,
                            e->n_features, false, &P, &err, true);
    if (st != QTS_OK) return fail(st, err);
    DevTables& T = e->bdev;
    int64_t tot = 0;
    st = up((Rec32**)&T.rec, P.rec32, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.path_leaf, P.path_leaf, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.path_zprod, P.path_zprod, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.path_val, P.path_val, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.slot_zexcl, P.slot_zexcl, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.slot_edge_begin, P.slot_edge_begin, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.edge_node, P.edge_node, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.edge_coef, P.edge_coef, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.empty_leaf, P.empty_leaf, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.pair_leaf2, P.pair_leaf2, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.pair_zprod2, P.pair_zprod2, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.pair_z, P.pair_z, &tot, "upload pair tables");
    if (st == QTS_OK) st = up(&T.pair_gslot, P.pair_gslot, &tot, "upload pair tables");
    if (st != QTS_OK) {
        release_batch_tables(e);
        return st;
    }
    T.bytes = tot;
    for (auto* v : {&P.path_zprod, &P.path_val, &P.slot_zexcl, &P.edge_coef, &P.pair_zprod2, &P.pair_z})
        std::vector<double>().swap(*v);
    for (auto* v : {&P.path_leaf, &P.slot_edge_begin, &P.edge_node, &P.pair_leaf2, &P.pair_gslot})
        std::vector<int64_t>().swap(*v);
    std::vector<Rec32>().swap(P.rec32);
    e->bready = true;
    return QTS_OK;
}

qts_status ensure_workspace(qts_ensemble* e, size_t bytes) {
    if (bytes <= e->work_bytes) return QTS_OK;
    if (e->d_work) {
        batch_forget(e);
        cudaError_t err = cudaDeviceSynchronize();
        if (err != cudaSuccess) return cuda_fail(err, "workspace resize sync");
        cudaFree(e->d_work);
        e->d_work = nullptr;
        e->work_bytes = 0;
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    cudaError_t err = cudaMalloc(&e->d_work, want);
    if (err != cudaSuccess) return cuda_fail(err, "workspace allocation");
    e->work_bytes = want;
    return QTS_OK;
}

// The device failure path on demand: one block waits, bounded, on an mbarrier
// that nothing arrives at; the wait runs out and latches QTS_ERR_TIMEOUT in the
// status word.  No copy is issued, so nothing is left in flight.
__global__ void wait_selftest_kernel(int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0)) report(status, QTS_ERR_TIMEOUT);
}

cudaError_t launch_wait_selftest(int* status, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(status);
    return cudaGetLastError();
}

qts_status check_call(qts_ensemble* e, const float* X, int64_t M, int32_t F, int32_t n_quad) {
    if (!e) return fail(QTS_ERR_ARG, "ensemble handle is NULL");
    if (F != e->n_features)
        return fail(QTS_ERR_ARG, "F = " + std::to_string(F) + " does not match the ensemble's " +
                                     std::to_string(e->n_features) + " features");
    if (M < 0) return fail(QTS_ERR_ARG, "M must be >= 0");
    if (M > 0 && !X) return fail(QTS_ERR_ARG, "X is NULL");
    if (M > ((int64_t)1 << 31)) return fail(QTS_ERR_UNSUPPORTED, "M above 2^31 samples");
    if (n_quad != QTS_NQ_EXACT && (n_quad < 1 || n_quad > QTS_MAX_QUAD))
        return fail(QTS_ERR_ARG, "n_quad must be QTS_NQ_EXACT or in [1, " + std::to_string(QTS_MAX_QUAD) + "]");
    return QTS_OK;
}

}  // namespace qts

using namespace qts;

extern "C" {

const char* qts_last_error(void) { return g_err.c_str(); }

qts_status qts_gauss_legendre(int32_t n, double* t, double* w) {
    if (!t || !w || n < 1 || n > 64) return fail(QTS_ERR_ARG, "n must be in [1, 64] and t, w non-NULL");
    return gauss_legendre(n, t, w) ? QTS_OK : fail(QTS_ERR_ARG, "gauss_legendre failed");
}

int32_t qts_exact_nodes(int32_t width, int32_t order) {
    if (width < 1 || width > QTS_MAX_UNIQUE_FEATURES_PER_PATH || order < 1) return 0;
    return exact_nodes(width, order);
}

static qts_status load_impl(int32_t n_trees, const int64_t* off, const int32_t* left,
                            const int32_t* right, const int32_t* feature, const float* threshold,
                            const uint8_t* default_left, const float* z, const float* leaf_value,
                            const uint8_t* is_cat, const uint64_t* cat_left, int32_t n_features,
                            uint32_t flags, qts_ensemble** out) {
    if (!out) return fail(QTS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_trees < 1 || !off || !left || !right || !feature || !threshold || !z || !leaf_value)
        return fail(QTS_ERR_ARG, "n_trees < 1 or a required array is NULL");
    if (n_features < 1 || n_features > QTS_MAX_FEATURES)
        return fail(QTS_ERR_UNSUPPORTED, "n_features must be in [1, " + std::to_string(QTS_MAX_FEATURES) + "]");
    if (flags & ~QTS_FLAG_FP64) return fail(QTS_ERR_ARG, "unknown flags");
    if (is_cat && !cat_left) return fail(QTS_ERR_ARG, "category_left_mask is NULL");
    for (int t = 0; t < n_trees; ++t)
        if (off[t + 1] <= off[t]) return fail(QTS_ERR_ARG, "tree_node_offsets must be increasing");
    if (off[0] != 0) return fail(QTS_ERR_ARG, "tree_node_offsets[0] must be 0");
    auto* e = new (std::nothrow) qts_ensemble();
    if (!e) return fail(QTS_ERR_OOM, "host allocation");
    const int64_t N = off[n_trees];
    e->n_trees = n_trees;
    e->n_features = n_features;
    e->n_nodes = N;
    e->flags = flags;
    cudaGetDevice(&e->device);
    e->off.assign(off, off + n_trees + 1);
    e->left.assign(left, left + N);
    e->right.assign(right, right + N);
    e->feature.assign(feature, feature + N);
    e->thr.assign(threshold, threshold + N);
    e->z.assign(z, z + N);
    e->leaf.assign(leaf_value, leaf_value + N);
    if (default_left) e->defl.assign(default_left, default_left + N);
    else e->defl.assign((size_t)N, 1);
    if (is_cat) {
        e->is_cat.assign(is_cat, is_cat + N);
        e->cat_left.assign(cat_left, cat_left + N);
    }
    std::string err;
    qts_status st = prepare(n_trees, e->off.data(), e->left.data(), e->right.data(),
                            e->feature.data(), e->thr.data(), e->defl.data(), e->z.data(),
                            e->leaf.data(), is_cat ? e->is_cat.data() : nullptr,
                            is_cat ? e->cat_left.data() : nullptr, n_features,
                            (flags & QTS_FLAG_FP64) != 0, &e->prep, &err);
    if (st != QTS_OK) {
        delete e;
        return fail(st, err);
    }
    cudaError_t ce = cudaMalloc(&e->d_status, sizeof(int));
    if (ce == cudaSuccess) ce = cudaMemset(e->d_status, 0, sizeof(int));
    if (ce != cudaSuccess) {
        delete e;
        return cuda_fail(ce, "status word");
    }
    st = upload(e);
    if (st != QTS_OK) {
        cudaFree(e->d_status);
        delete e;
        return st;
    }
    for (int D = 0; D <= kMaxD; ++D) e->tune[D] = default_tune(std::max(D, 1));
    *out = e;
    return QTS_OK;
}

qts_status qts_load_ensemble(int32_t n_trees, const int64_t* off, const int32_t* left,
                             const int32_t* right, const int32_t* feature, const float* threshold,
                             const uint8_t* default_left, const float* z, const float* leaf_value,
                             int32_t n_features, uint32_t flags, qts_ensemble** out) {
    return load_impl(n_trees, off, left, right, feature, threshold, default_left, z, leaf_value,
                     nullptr, nullptr, n_features, flags, out);
}

qts_status qts_load_ensemble_cat(int32_t n_trees, const int64_t* off, const int32_t* left,
                                 const int32_t* right, const int32_t* feature, const float* threshold,
                                 const uint8_t* default_left, const float* z, const float* leaf_value,
                                 const uint8_t* is_categorical, const uint64_t* category_left_mask,
                                 int32_t n_features, uint32_t flags, qts_ensemble** out) {
    return load_impl(n_trees, off, left, right, feature, threshold, default_left, z, leaf_value,
                     is_categorical, category_left_mask, n_features, flags, out);
}

qts_status qts_update_params(qts_ensemble* e, const float* z, const float* leaf_value) {
    if (!e || !z || !leaf_value) return fail(QTS_ERR_ARG, "NULL argument");
    std::vector<float> z0 = e->z, l0 = e->leaf;
    e->z.assign(z, z + e->n_nodes);
    e->leaf.assign(leaf_value, leaf_value + e->n_nodes);
    Prepared P;
    std::string err;
    const bool cat = !e->is_cat.empty();
    qts_status st = prepare(e->n_trees, e->off.data(), e->left.data(), e->right.data(),
                            e->feature.data(), e->thr.data(), e->defl.data(), e->z.data(),
                            e->leaf.data(), cat ? e->is_cat.data() : nullptr,
                            cat ? e->cat_left.data() : nullptr, e->n_features,
                            (e->flags & QTS_FLAG_FP64) != 0, &P, &err);
    if (st != QTS_OK) {
        e->z = z0;
        e->leaf = l0;
        return fail(st, err);
    }
    cudaError_t ce = cudaDeviceSynchronize();
    if (ce != cudaSuccess) return cuda_fail(ce, "update sync");
    batch_forget(e);
    release_device(e);
    e->prep = std::move(P);
    return upload(e);
}

qts_status qts_shap_values(qts_ensemble* e, const float* X, int64_t M, int32_t F, int32_t n_quad,
                           double* phi, qts_stream_t stream) {
    qts_status st = check_call(e, X, M, F, n_quad);
    if (st != QTS_OK) return st;
    if (M == 0) return QTS_OK;
    if (!phi) return fail(QTS_ERR_ARG, "phi is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    // FP32 runs on the pair tables (built on the first call that needs them)
    const bool fp64 = (e->flags & QTS_FLAG_FP64) != 0;
    if (!fp64) {
        st = ensure_batch_tables(e);
        if (st != QTS_OK) return st;
    }
    const Prepared& P = fp64 ? e->prep : e->bprep;
    cudaError_t ce = launch_phi_init(phi, M, F, P.bias, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "phi init launch");
    for (const Bucket& b : P.buckets) {
        // the bucket's rule, padded to whole node pairs (QTS_NQ_EXACT: ceil(D/2) points)
        QuadF qf;
        QuadD qd;
        if (!make_quad(nodes_for(n_quad, b.D, 1), &qf, &qd, 2)) return fail(QTS_ERR_ARG, "quadrature rule");
        ce = launch_fwd_bucket(e, b, X, M, F, qf, qd, phi, e->tune[b.D], s);
        if (ce != cudaSuccess) return cuda_fail(ce, "forward kernel launch");
    }
    return QTS_OK;
}

qts_status qts_selftest_wait_timeout(qts_ensemble* e, qts_stream_t stream) {
    if (!e) return fail(QTS_ERR_ARG, "ensemble handle is NULL");
    cudaError_t ce = launch_wait_selftest(e->d_status, (cudaStream_t)stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "self-test launch");
    return QTS_OK;
}

qts_status qts_sync_status(qts_ensemble* e, qts_stream_t stream) {
    if (!e) return fail(QTS_ERR_ARG, "ensemble handle is NULL");
    cudaError_t ce = cudaStreamSynchronize((cudaStream_t)stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "stream synchronize");
    int h = 0;
    ce = cudaMemcpy(&h, e->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_fail(ce, "status read");
    if (h != 0) {
        cudaMemset(e->d_status, 0, sizeof(int));
        return fail((qts_status)h, h == QTS_ERR_TIMEOUT ? "a bounded device wait ran out"
                                                        : "device-side check failed");
    }
    return QTS_OK;
}

qts_status qts_get_info(const qts_ensemble* e, qts_info* out) {
    if (!e || !out) return fail(QTS_ERR_ARG, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->n_trees = e->n_trees;
    out->n_features = e->n_features;
    out->n_nodes = e->n_nodes;
    out->n_leaves = e->prep.n_leaves;
    out->n_paths = e->prep.n_paths;
    out->max_unique = e->prep.max_unique;
    out->sum_unique = e->prep.sum_unique;
    out->n_buckets = (int32_t)e->prep.buckets.size();
    for (size_t i = 0; i < e->prep.buckets.size() && i < 32; ++i) {
        out->bucket_width[i] = e->prep.buckets[i].D;
        out->bucket_paths[i] = e->prep.buckets[i].n_paths;
    }
    out->expected_value = e->prep.bias;
    out->device_bytes = e->device_bytes;
    out->flags = e->flags;
    return QTS_OK;
}

qts_status qts_describe_ensemble(int32_t n_trees, const int64_t* off, const int32_t* left,
                                 const int32_t* right, const int32_t* feature, const float* threshold,
                                 const uint8_t* default_left, const float* z, const float* leaf_value,
                                 int32_t n_features, uint32_t flags, qts_info* out) {
    if (!out || n_trees < 1 || !off || !left || !right || !feature || !threshold || !z || !leaf_value)
        return fail(QTS_ERR_ARG, "NULL argument or n_trees < 1");
    if (n_features < 1 || n_features > QTS_MAX_FEATURES)
        return fail(QTS_ERR_UNSUPPORTED, "n_features out of range");
    for (int t = 0; t < n_trees; ++t)
        if (off[t + 1] <= off[t]) return fail(QTS_ERR_ARG, "tree_node_offsets must be increasing");
    std::vector<uint8_t> defl;
    if (!default_left) defl.assign((size_t)off[n_trees], 1);
    Prepared P;
    std::string err;
    const bool fp64 = (flags & QTS_FLAG_FP64) != 0;
    const bool pairs = (flags & QTS_DESCRIBE_PAIRS) != 0;
    qts_status st = prepare(n_trees, off, left, right, feature, threshold,
                            default_left ? default_left : defl.data(), z, leaf_value, nullptr, nullptr,
                            n_features, fp64, &P, &err, pairs);
    if (st != QTS_OK) return fail(st, err);
    std::memset(out, 0, sizeof(*out));
    out->n_trees = n_trees;
    out->n_features = n_features;
    out->n_nodes = off[n_trees];
    out->n_leaves = P.n_leaves;
    out->n_paths = P.n_paths;
    out->max_unique = P.max_unique;
    out->sum_unique = P.sum_unique;
    out->n_buckets = (int32_t)P.buckets.size();
    for (size_t i = 0; i < P.buckets.size() && i < 32; ++i) {
        out->bucket_width[i] = P.buckets[i].D;
        out->bucket_paths[i] = P.buckets[i].n_paths;
    }
    out->expected_value = P.bias;
    out->device_bytes = (int64_t)((fp64 ? P.rec64.size() * sizeof(Rec64) : P.rec32.size() * sizeof(Rec32)) +
                                  P.path_leaf.size() * 8 + P.path_zprod.size() * 8 +
                                  P.slot_edge_begin.size() * 8 + P.edge_node.size() * 16);
    out->flags = flags;
    return QTS_OK;
}

qts_status qts_describe_paths(int32_t n_trees, const int64_t* off, const int32_t* left, const int32_t* right,
                              const int32_t* feature, const float* threshold, const uint8_t* default_left,
                              const float* z, const float* leaf_value, const uint8_t* is_categorical,
                              const uint64_t* category_left_mask, int32_t n_features, int64_t* n_records,
                              int64_t* n_paths, uint32_t* records, int64_t* path_leaf, int32_t* path_width) {
    if (!n_records || !n_paths || n_trees < 1 || !off || !left || !right || !feature || !threshold || !z ||
        !leaf_value)
        return fail(QTS_ERR_ARG, "NULL argument or n_trees < 1");
    if (n_features < 1 || n_features > QTS_MAX_FEATURES)
        return fail(QTS_ERR_UNSUPPORTED, "n_features out of range");
    if (is_categorical && !category_left_mask) return fail(QTS_ERR_ARG, "category_left_mask is NULL");
    for (int t = 0; t < n_trees; ++t)
        if (off[t + 1] <= off[t]) return fail(QTS_ERR_ARG, "tree_node_offsets must be increasing");
    std::vector<uint8_t> defl;
    if (!default_left) defl.assign((size_t)off[n_trees], 1);
    Prepared P;
    std::string err;
    qts_status st = prepare(n_trees, off, left, right, feature, threshold,
                            default_left ? default_left : defl.data(), z, leaf_value, is_categorical,
                            category_left_mask, n_features, false, &P, &err);
    if (st != QTS_OK) return fail(st, err);
    *n_records = (int64_t)P.rec32.size();
    *n_paths = P.n_paths;
    if (!records) return QTS_OK;
    if (!path_leaf || !path_width) return fail(QTS_ERR_ARG, "path_leaf or path_width is NULL");
    std::memcpy(records, P.rec32.data(), P.rec32.size() * sizeof(Rec32));
    std::memcpy(path_leaf, P.path_leaf.data(), P.path_leaf.size() * sizeof(int64_t));
    for (const Bucket& b : P.buckets)
        for (int64_t p = 0; p < b.n_paths; ++p) path_width[b.path_base + p] = b.D;
    return QTS_OK;
}

void qts_free(qts_ensemble* e) {
    if (!e) return;
    batch_forget(e);
    cudaDeviceSynchronize();
    release_device(e);
    cudaFree(e->d_status);
    cudaFree(e->d_work);
    delete e;
}

}  // extern "C"
