// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "qtreeshap.h"

// Heavy translation units are compiled in parts, in parallel: a file whose
// first lines say "qts-build-parts: N" is compiled N times with -DQTS_PART=k.
// Part 0 holds the host code and sees only declarations of the per-width
// launchers; part k >= 1 defines the kernels and instantiates its share of the
// launchers.  Compiled without QTS_PART, a file is one complete unit.
#ifdef QTS_PART
#define QTS_HOST_PART (QTS_PART == 0)
#define QTS_DEVICE_PARTS (QTS_PART != 0)
#define QTS_IN_PART(k) (QTS_PART == (k))
#else
#define QTS_HOST_PART 1
#define QTS_DEVICE_PARTS 1
#define QTS_IN_PART(k) 1
#endif

namespace qts {

// ---------------------------------------------------------------- records --
//
// FP32 path table of a bucket of width D: each path occupies D+1 consecutive
// 16-byte records.  Record 0 is the header {val, prod_j z_j, 0, 0}; records
// 1..D are the merged elements {z, lo, hi, bits} with bits = feature index
// (low 24 bits) | NaN-satisfies flag (bit 31).  Paths with d < D unique
// features are padded with neutral elements {1, -inf, +inf, F | NaN-ok}:
// a = 1 at every node and o - z = 0, so they add nothing.  Elements are sorted
// by feature index, so element order = feature order (used by interactions).
struct __align__(16) Rec32 {
    float z, lo, hi;
    uint32_t bits;
};
constexpr uint32_t kNanOk = 0x80000000u;
// Categorical element: lo and hi hold the low and high 32 bits of the set of
// categories that satisfy every split merged into it, kOtherOk says whether a
// value that is not a category (outside [0, 64)) satisfies them.
constexpr uint32_t kCat = 0x40000000u;
constexpr uint32_t kOtherOk = 0x20000000u;
constexpr uint32_t kFeatMask = 0x00FFFFFFu;
// Sibling-pair element (pair tables of the batched pass; always the path's last
// record).  Leaves A (left) and B (right) of a numerical split at threshold
// theta share every other element; this one has z = alpha = val_A z_A +
// val_B z_B and [lo, hi) = the interval of the splits on the feature above the
// pair, and a sample x gives d = (x in [lo, hi) ? (x < theta ? dA : dB) : -alpha)
// (NaN: kNanOk and kDefLeft choose).  The path header holds {1 (val), dA =
// val_A - alpha, dB = val_B - alpha, bits of theta}.
constexpr uint32_t kPairElem = 0x10000000u;
constexpr uint32_t kDefLeft = 0x08000000u;

// FP64 table: 32-byte records {z, 0, lo, hi, bits, 0}; header {val, prod z}.
struct __align__(16) Rec64 {
    double z;
    double aux;
    float lo, hi;
    uint32_t bits;
    uint32_t pad;
};

constexpr int kMaxBuckets = 32;
constexpr int kMaxD = QTS_MAX_UNIQUE_FEATURES_PER_PATH;

// bucket widths: exact up to 16 unique features, then steps of 4 and 8
int bucket_width_for(int d);

struct Bucket {
    int D = 0;              // record width (unique features, padded)
    int64_t n_paths = 0;
    int64_t rec_off = 0;    // first record (Rec32 or Rec64 units) in d_rec
    int64_t path_base = 0;  // global path index of the first path
    int64_t slot_base = 0;  // global element slot of the first element (n_paths * D slots)
};

// Host result of path preparation (Sec. 2 merging).
struct Prepared {
    std::vector<Bucket> buckets;
    std::vector<Rec32> rec32;     // FP32 tables, all buckets back to back
    std::vector<Rec64> rec64;     // FP64 tables (QTS_FLAG_FP64 only)
    std::vector<int64_t> path_leaf;   // per global path: leaf node (global index)
    std::vector<double> path_zprod;   // per global path: prod_j z_j (fp64)
    std::vector<double> path_val;     // per global path: leaf value
    std::vector<double> slot_zexcl;        // per element slot: prod_{l != j} z_l of its path
    std::vector<int64_t> slot_edge_begin;  // per element slot + 1: CSR into edge arrays
    std::vector<int64_t> edge_node;        // global node index of the merged edge
    std::vector<double> edge_coef;         // prod of the other edge weights in the element
    std::vector<int64_t> empty_leaf;       // leaves of single-leaf trees (no split)
    std::vector<double> empty_val;
    int64_t n_paths = 0, n_slots = 0, n_leaves = 0, sum_unique = 0;
    int max_unique = 0;
    double bias = 0.0;  // E[f]
    bool has_cat = false;  // some element is categorical: kernels take their NaN-aware variant
    // pair tables (sibling leaves of a numerical split as one path, kPairElem)
    bool pairs = false;
    int64_t n_pair_paths = 0;
    std::vector<int64_t> pair_leaf2;   // per path: leaf B of a pair, -1 otherwise (path_leaf is A)
    std::vector<double> pair_zprod2;   // per path: prod of leaf B's merged z (path_zprod is A's)
    std::vector<double> pair_z;        // per path: z_A, z_B of the pair element
    std::vector<int64_t> pair_gslot;   // per path: slot of the pair element, -1 otherwise
};

// Prepare the path tables (host, multi-threaded).  Returns QTS_OK or an error
// with the message in *err.
qts_status prepare(int32_t n_trees, const int64_t* off, const int32_t* left, const int32_t* right,
                   const int32_t* feature, const float* thr, const uint8_t* defl, const float* z,
                   const float* leaf, const uint8_t* is_cat, const uint64_t* cat_left, int32_t F,
                   bool fp64, Prepared* out, std::string* err, bool pairs = false);

// Gauss-Legendre nodes on [0,1] (Golub-Welsch via Jacobi eigen-decomposition).
bool gauss_legendre(int n, double* t, double* w);

// Device copies of one set of path tables and the adjoint's metadata.
struct DevTables {
    void* rec = nullptr;               // Rec32 records
    int64_t* path_leaf = nullptr;
    double* path_zprod = nullptr;
    double* path_val = nullptr;
    double* slot_zexcl = nullptr;
    int64_t* slot_edge_begin = nullptr;
    int64_t* edge_node = nullptr;
    double* edge_coef = nullptr;
    int64_t* empty_leaf = nullptr;
    int64_t* pair_leaf2 = nullptr;     // pair tables only
    double* pair_zprod2 = nullptr;
    double* pair_z = nullptr;
    int64_t* pair_gslot = nullptr;
    int64_t bytes = 0;
};

// Launch tuning of one bucket width.
struct Tune {
    int warps = 4;        // warps per block (samples are shared, paths split)
    int paths = 128;      // paths per block (chunk)
    int sub = 32;         // paths per staged sub-chunk
    int np = 8;           // nodes per register pass (8, 4 or 2)
    int bpaths = 128;     // paths per work item of the fused forward + adjoint pass
    int priv = 1;         // forward: 1 each warp owns a sample tile (when it fits), 2 the
                          // warps share one and split the paths with a phi tile each,
                          // 0 they share one phi tile (shared-memory atomics)
    // choices of the batched-launch tuner (0: not tuned, the launch's default)
    int bt_paths = 0;     // paths per work item of the persistent batched kernel
    int bt_mode = 0;      // sample mapping of the packed fused pass: 2 (64 samples
                          // per warp) or 3 (64 samples shared by the block's warps)
    int bt_occ = 0;       // blocks per SM of the width's register class (0: as many as
                          // fit; fewer leave more of the SM's shared memory to L1)
};

}  // namespace qts

// The opaque handle.
struct qts_ensemble {
    int32_t n_trees = 0, n_features = 0;
    int64_t n_nodes = 0;
    uint32_t flags = 0;
    int device = 0;
    // host copy of the model (for qts_update_params)
    std::vector<int64_t> off;
    std::vector<int32_t> left, right, feature;
    std::vector<float> thr, z, leaf;
    std::vector<uint8_t> defl;
    std::vector<uint8_t> is_cat;      // empty: no categorical splits
    std::vector<uint64_t> cat_left;
    // prepared tables
    qts::Prepared prep;
    // device memory
    void* d_rec = nullptr;            // Rec32 or Rec64 tables
    int64_t* d_path_leaf = nullptr;   // n_paths
    double* d_path_zprod = nullptr;   // n_paths
    double* d_path_val = nullptr;     // n_paths
    double* d_slot_zexcl = nullptr;   // n_slots
    int64_t* d_slot_edge_begin = nullptr;  // n_slots + 1
    int64_t* d_edge_node = nullptr;
    double* d_edge_coef = nullptr;
    int64_t* d_empty_leaf = nullptr;
    int* d_status = nullptr;          // device status word
    int64_t device_bytes = 0;
    // grow-only workspace (interaction accumulators, adjoint per-path sums)
    void* d_work = nullptr;
    size_t work_bytes = 0;
    // depth-first (Algorithm 1) program: preorder records of the internal
    // nodes, built on the first call that needs it
    void* d_dfs = nullptr;
    int64_t* d_dfs_off = nullptr;     // per tree, n_trees + 1
    int dfs_levels = 0;               // internal-node depth + 1
    int64_t dfs_records = 0;
    // pair tables of the batched pass (sibling leaves merged), built on the
    // first batched call that includes this ensemble
    qts::Prepared bprep;
    qts::DevTables bdev;
    bool bready = false;
    // per-width launch tuning (index = bucket width)
    qts::Tune tune[qts::kMaxD + 1];
    bool tuned = false;
    uint32_t tune_gen = 0;            // bumped by every tuning call (cached batched graphs key on it)
};

namespace qts {

void set_error(const std::string& msg);
qts_status fail(qts_status st, const std::string& msg);
qts_status cuda_fail(cudaError_t e, const char* what);
qts_status ensure_workspace(qts_ensemble* e, size_t bytes);
qts_status upload(qts_ensemble* e);
void release_device(qts_ensemble* e);
void release_dfs(qts_ensemble* e);      // drop the depth-first program (rebuilt on demand)
qts_status ensure_batch_tables(qts_ensemble* e);  // build the pair tables of the batched pass
void release_batch_tables(qts_ensemble* e);
int num_sms();
void batch_forget(const qts_ensemble* e);  // drop cached batched graphs using e

// GL nodes packed for the kernels (fp32 and fp64), padded to a multiple of 8
// with zero-weight nodes at t = 1/2.
struct QuadF {
    float t[QTS_MAX_QUAD + 8];
    float w[QTS_MAX_QUAD + 8];
    int n, n_pad;
};
struct QuadD {
    double t[QTS_MAX_QUAD + 8];
    double w[QTS_MAX_QUAD + 8];
    int n, n_pad;
};
// n nodes, padded with zero-weight nodes to a multiple of `pad` (the node
// count of one register pass of the kernel that takes the rule)
bool make_quad(int n, QuadF* qf, QuadD* qd, int pad = 8);

// Points that integrate an order-s quantity exactly on paths of at most
// `width` unique features: ceil((width - s + 1) / 2), at least 1 (Thm 2).
inline int exact_nodes(int width, int order) {
    const int deg = width - order;  // degree of the integrand
    return deg < 1 ? 1 : deg / 2 + 1;
}
// The points an n_quad argument asks for on paths of `width` unique features.
inline int nodes_for(int n_quad, int width, int order) {
    return n_quad == QTS_NQ_EXACT ? exact_nodes(width, order) : n_quad;
}

// validate common call arguments
qts_status check_call(qts_ensemble* e, const float* X, int64_t M, int32_t F, int32_t n_quad);

// ----------------------------------------------------- kernel launchers ---
// (defined in the .cu files; all enqueue on `st` and return cudaGetLastError)

cudaError_t launch_phi_init(double* phi, int64_t M, int F, double bias, cudaStream_t st);
cudaError_t launch_wait_selftest(int* status, cudaStream_t st);
cudaError_t launch_fwd_bucket(const qts_ensemble* e, const Bucket& b, const float* X, int64_t M,
                              int F, const QuadF& q, const QuadD& qd, double* phi, const Tune& tn,
                              cudaStream_t st);
// pairs: b is a bucket of the sibling-pair tables (e->bprep), else of e->prep
cudaError_t launch_int_bucket(const qts_ensemble* e, const Bucket& b, bool pairs, const float* X, int64_t M,
                              int F, const QuadF& q, double* acc_pair, double* acc_phi,
                              cudaStream_t st);
cudaError_t launch_int_finalize(const double* acc_pair, const double* acc_phi, int64_t M, int F,
                                double bias, float* out, cudaStream_t st);
cudaError_t launch_bwd_bucket(const qts_ensemble* e, const Bucket& b, const float* X,
                              const float* grad, int64_t M, int F, const QuadF& q,
                              double* g_val, double* g_slot, double* phi, const Tune& tn,
                              cudaStream_t st);
cudaError_t launch_bwd_epilogue(const qts_ensemble* e, const float* grad, int64_t M, int F,
                                const double* g_val, const double* g_slot, double* d_leaf,
                                double* d_z, double* g_bias_scratch, cudaStream_t st);
// the same for the pair tables of the batched pass (two g_val sums per path)
cudaError_t launch_bwd_epilogue_pairs(const qts_ensemble* e, const float* grad, int64_t M, int F,
                                      const double* g_val, const double* g_slot, double* d_leaf,
                                      double* d_z, double* g_bias_scratch, cudaStream_t st);

}  // namespace qts
