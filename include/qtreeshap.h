/*
 * qtreeshap.h - C ABI of the GB300 (sm_103a) Quadrature-TreeSHAP library.
 *
 * What it computes (arXiv 2605.04497):
 *   For a tree ensemble with edge weights w_e = n_child/n_parent (Sec. 2) and a
 *   sample x, the Path-Dependent Shapley value of feature i is
 *       phi_i = sum_v val(v) (o_i - z_i) int_0^1 prod_{j != i} a_j(p) dp
 *   and the pairwise Shapley interaction index of features i != j is
 *       SII_ij = sum_v val(v) (o_i - z_i)(o_j - z_j) int_0^1 prod_{k != i,j} a_k(p) dp,
 *   where the sum runs over leaves v whose root-to-leaf path uses the features,
 *   the path's splits are merged per feature (Eq. q_def), z_j is the product of
 *   the path's edge weights on feature j, o_j = 1 if x satisfies all of the
 *   path's splits on j, and a_j(p) = (1-p) z_j + p o_j.  This is Thm 1 with
 *   S = {i} and S = {i,j} (Eq. weighted_banzhaf_iv_v2 with R_empty = val prod w,
 *   q_j = o_j/z_j) integrated over p as in Eq. ao_shap_is_intergral_of_ao_banzhaf.
 *   The integral is evaluated with n_quad Gauss-Legendre points on [0,1]
 *   (Eq. shap_as_weighted_banzhafs; Sec. 6 fixes n = 8), which is exact when
 *   the path has at most 2*n_quad unique features (Thm 2).
 *
 * Conventions (all entry points):
 *   - Device pointers are CUDA device memory of the current device; they are
 *     owned by the caller and must stay valid until the stream work completes.
 *     Host pointers are read during the call only.
 *   - Every compute call is asynchronous on `stream` and only enqueues work.
 *     Argument errors are reported synchronously by the return code; faults
 *     detected on the device (a bounded wait that ran out) are latched in the
 *     ensemble's device status word and reported by qts_sync_status.
 *   - Nothing ever aborts or traps; on error the return code is non-zero and
 *     qts_last_error() describes it (thread-local string).
 *   - Calls that use the same ensemble must not overlap on the GPU (they share
 *     the ensemble's workspace); enqueue them on one stream.
 *   - X is M x F row-major fp32 with F equal to the ensemble's n_features.
 *     x[f] < threshold goes left, x[f] >= threshold right, NaN goes the node's
 *     default direction (categorical splits: see qts_load_ensemble_cat).
 */
#ifndef QTREESHAP_H
#define QTREESHAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *qts_stream_t; /* same handle as cudaStream_t; NULL = legacy default */

typedef struct qts_ensemble qts_ensemble; /* opaque; owns the device path tables */

typedef enum qts_status {
    QTS_OK = 0,
    QTS_ERR_ARG = 1,          /* invalid argument (pointer, size, topology) */
    QTS_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    QTS_ERR_OOM = 3,          /* device or host allocation failed */
    QTS_ERR_UNSUPPORTED = 4,  /* valid input outside the supported envelope */
    QTS_ERR_TIMEOUT = 5,      /* a bounded device wait ran out (reported by qts_sync_status) */
    QTS_ERR_DEVICE_CHECK = 6  /* a device-side consistency check failed */
} qts_status;

/* flags for qts_load_ensemble */
#define QTS_FLAG_FP64 1u /* all path arithmetic in FP64 (correctness mode, slow on GB300) */

/* Limits of the supported envelope. */
#define QTS_MAX_UNIQUE_FEATURES_PER_PATH 64
#define QTS_MAX_FEATURES 832 /* the kernels keep a sample tile and an accumulator tile of F + 1
                                rows in shared memory (F = 784: Fashion-MNIST-shaped models) */
#define QTS_MAX_QUAD 32
/* n_quad = QTS_NQ_EXACT: per bucket of paths with at most w unique features,
   the fewest Gauss-Legendre points that make an order-s quantity exact,
   ceil((w - s + 1) / 2) (Thm 2; qts_exact_nodes).  The first-order, adjoint and
   batched calls and pairwise interactions choose it per bucket, so short
   paths take fewer points than long ones; interactions of order >= 3 and the
   depth-first call choose it once, from the ensemble's widest path.  Unlike a fixed n_quad it is exact for every width
   up to QTS_MAX_UNIQUE_FEATURES_PER_PATH (32 points at width 64). */
#define QTS_NQ_EXACT 0
#define QTS_MAX_FEATURES_ORDER3 128
#define QTS_MAX_CATEGORIES 64 /* categories 0..63 of a categorical split */

/*
 * qts_load_ensemble - copy a tree ensemble and build its path tables.
 * Sec. 2 (edge weights, Eq. R_empty, Eq. q_def): every root-to-leaf path is
 * enumerated, splits on the same feature are merged into one element
 * (z = product of their edge weights, the interval [lo, hi) satisfying them all,
 * and whether NaN satisfies them all), paths are bucketed by unique-feature
 * count and uploaded as structure-of-arrays tables.
 *
 *   n_trees            number of trees (>= 1)
 *   tree_node_offsets  host, n_trees+1 ascending; tree t owns nodes
 *                      [off[t], off[t+1]); its root is local node 0
 *   left, right        host, local child indices within the tree, -1 at leaves
 *                      (both -1 or both >= 0); children after their parent is
 *                      not required, but every tree must be a proper binary tree
 *   feature            host, split feature in [0, n_features) (ignored at leaves)
 *   threshold          host, fp32 split value
 *   default_left       host, 1 if NaN goes left (may be NULL: NaN goes left)
 *   z                  host, edge weight into the node (root ignored); a cover
 *                      fraction in (0, 1], but any positive finite value is
 *                      accepted so that refits may move it
 *   leaf_value         host, value at leaves (ignored at internal nodes)
 *   n_features         number of features F, 1..QTS_MAX_FEATURES
 *   flags              0 or QTS_FLAG_FP64
 *   out                receives the handle; free with qts_free
 * Errors: QTS_ERR_ARG (bad pointers/topology/z), QTS_ERR_UNSUPPORTED (a path
 * with more than QTS_MAX_UNIQUE_FEATURES_PER_PATH unique features), QTS_ERR_OOM,
 * QTS_ERR_CUDA.  Synchronous (uploads with cudaMemcpy on the current device).
 */
qts_status qts_load_ensemble(int32_t n_trees, const int64_t *tree_node_offsets,
                             const int32_t *left, const int32_t *right, const int32_t *feature,
                             const float *threshold, const uint8_t *default_left, const float *z,
                             const float *leaf_value, int32_t n_features, uint32_t flags,
                             qts_ensemble **out);

/*
 * qts_load_ensemble_cat - qts_load_ensemble for ensembles with categorical
 * splits (the paper's Adult models carry XGBoost categorical splits, Sec. 8).
 * A categorical split on feature f sends x left iff x[f] is not NaN,
 * 0 <= x[f] < QTS_MAX_CATEGORIES and bit floor(x[f]) of its mask is set; NaN
 * follows default_left, every other value goes right.  Along a path the splits
 * on one feature intersect (Eq. q_def: q_i depends on all splits on i), so a
 * merged element holds the set of categories that satisfies all of them.
 *   is_categorical       host, one per node: 1 if the node's split is
 *                        categorical (ignored at leaves); NULL = none
 *   category_left_mask   host, one per node: the categories that go left
 *                        (ignored unless is_categorical); may be NULL only if
 *                        is_categorical is NULL
 *   other arguments      as qts_load_ensemble
 * Errors: as qts_load_ensemble, plus QTS_ERR_ARG when a feature has both
 * numerical and categorical splits in the ensemble.  Every entry point except
 * qts_shap_values_alg1 (QTS_ERR_UNSUPPORTED) accepts such an ensemble;
 * qts_update_params keeps the split types and masks.
 */
qts_status qts_load_ensemble_cat(int32_t n_trees, const int64_t *tree_node_offsets,
                                 const int32_t *left, const int32_t *right, const int32_t *feature,
                                 const float *threshold, const uint8_t *default_left, const float *z,
                                 const float *leaf_value, const uint8_t *is_categorical,
                                 const uint64_t *category_left_mask, int32_t n_features,
                                 uint32_t flags, qts_ensemble **out);

/*
 * qts_update_params - replace edge weights and leaf values (same topology) and
 * rebuild the path tables (Sec. 2).  z, leaf_value: host, one entry per node.
 * Synchronous.  The sibling-pair tables of the FP32 calls are dropped and built
 * again on the next call that needs them.  Errors as qts_load_ensemble.
 */
qts_status qts_update_params(qts_ensemble *ens, const float *z, const float *leaf_value);

/*
 * qts_shap_values - first-order Shapley values (Thm 1 with S = {i}, Eq.
 * shap_as_weighted_banzhafs, Alg. 1 with s = 1).
 *   X       device, M x F fp32 row-major
 *   M       samples (>= 0; 0 is a no-op), F must equal the ensemble's n_features
 *   n_quad  Gauss-Legendre points, 1..QTS_MAX_QUAD (8 is the fast path), or
 *           QTS_NQ_EXACT: ceil(w / 2) points for the paths of width w
 *   phi     device, M x (F+1) fp64, overwritten; phi[s][F] = E[f] = sum_v R_empty^v
 *           (the bias, so that sum_f phi[s][f] = f(x_s))
 * Per-path arithmetic is FP32 (FP64 with QTS_FLAG_FP64); contributions are
 * accumulated in FP32 over at most a few thousand paths, then in FP64 across
 * path chunks and trees.  With M <= 16 lanes are (path, sample) pairs instead
 * of one sample per lane.
 * FP32 ensembles run on a second set of path tables in which each pair of
 * sibling leaves of a numerical split is one path (see qts_get_batch_info);
 * it is built by the first FP32 forward, adjoint or batched call (host
 * preparation, cudaMalloc and synchronous copies, about 60% more device memory
 * than the per-leaf tables), so that first call must not be inside a stream
 * capture; later calls only enqueue on `stream`.
 */
qts_status qts_shap_values(qts_ensemble *ens, const float *X, int64_t M, int32_t F,
                           int32_t n_quad, double *phi, qts_stream_t stream);

/*
 * qts_shap_values_alg1 - the same first-order Shapley values as qts_shap_values,
 * computed by the depth-first traversal of Algorithm 1 (Sec. 5) instead of
 * per-path products.  Each tree is walked once per sample: the products of the
 * ancestors' merged factors a_f(t) = z_f + (o_f - z_f) t (Thm 1) at the
 * quadrature nodes travel down, the subtrees' leaf sums travel up, and an edge
 * on a feature already split on above it is telescoped against that ancestor
 * (Eq. our_telescoping_background).  The work grows with the number of edges,
 * not with the summed path lengths, which pays for deep trees whose paths share
 * long prefixes.
 *   Arguments, output layout and ownership as qts_shap_values (X device M x F
 *   fp32 row-major; phi device M x (F+1) fp64, overwritten, phi[s][F] = E[f]).
 *   Accumulation: FP32 over a chunk of trees per 32-sample tile, FP64 across
 *   chunks.
 * Errors: as qts_shap_values, plus QTS_ERR_UNSUPPORTED for an ensemble loaded
 * with QTS_FLAG_FP64, for internal nodes more than 62 levels deep, or when the
 * per-warp shared memory (about 2 KiB per tree level plus 260 bytes per
 * feature) exceeds one block.  The first call on an ensemble (and the first
 * after qts_update_params) builds the traversal program on the host and uploads
 * it with cudaMalloc and a synchronous cudaMemcpy, so it must not be the first
 * call inside a stream capture; later calls only enqueue on `stream`.
 * QTS_NQ_EXACT takes ceil(d / 2) points for the ensemble's widest path d.
 */
qts_status qts_shap_values_alg1(qts_ensemble *ens, const float *X, int64_t M, int32_t F,
                                int32_t n_quad, double *phi, qts_stream_t stream);

/*
 * qts_shap_interactions - pairwise Shapley interaction values (Thm 1 with
 * S = {i,j}; Alg. 1 with s = 2) in the pred_interactions layout:
 *   phi_ij  device, M x (F+1) x (F+1) fp32, overwritten:
 *           [s][i][j] = SII_ij / 2 for i != j < F,
 *           [s][i][i] = phi_i - sum_{j != i} SII_ij / 2 (rows sum to phi_i),
 *           [s][F][F] = E[f], other entries of row/column F are 0.
 * Cross-tree accumulation is FP64 in the ensemble's workspace (device memory
 * of M * (F(F+1)/2) doubles, grown on demand with cudaMalloc).  Runs on the
 * sibling-pair tables of qts_shap_values (each pair's element is one more
 * linear factor of every pair term; built by the first call that needs them,
 * so that call must not be inside a stream capture).  n_quad as
 * qts_shap_values; QTS_NQ_EXACT takes ceil(D / 2) points per bucket of width
 * D (the pair terms need ceil((D - 1) / 2), the diagonal's first-order values
 * ceil(D / 2)).
 */
qts_status qts_shap_interactions(qts_ensemble *ens, const float *X, int64_t M, int32_t F,
                                 int32_t n_quad, float *phi_ij, qts_stream_t stream);

/*
 * qts_shap_interactions3 - third-order Shapley interaction indices (Thm 1 with
 * S = {i, j, k}; Alg. 1 with s = 3; the paper's any-order construction):
 *   SII_ijk = sum_v val (o_i - z_i)(o_j - z_j)(o_k - z_k) int_0^1 prod_{l not in {i,j,k}} a_l(p) dp
 * n_quad points are exact for paths of at most 2 n_quad + 2 unique features
 * (Thm 2).  Output, compact and symmetric-free:
 *   sii3   device, M x C(F,3) fp32, overwritten; entry [s][t] for the triple
 *          a < b < c with t = (C(F,3) - C(F-a,3)) + (C(F-a-1,2) - C(F-b,2)) + (c-b-1)
 * Cross-path accumulation is FP64 in the ensemble's workspace (C(F,3) * M
 * doubles, grown on demand with cudaMalloc).  F <= QTS_MAX_FEATURES_ORDER3,
 * paths of at most 16 unique features, FP32 tables only.
 */
qts_status qts_shap_interactions3(qts_ensemble *ens, const float *X, int64_t M, int32_t F,
                                  int32_t n_quad, float *sii3, qts_stream_t stream);

/*
 * qts_shap_interactions_order - Shapley interaction indices of any order s,
 * 2 <= s <= 8 (Thm 1 with |S| = s; Alg. 1 with general s; the paper times
 * orders 2-6, Sec. 8).  For every merged path containing all features of S,
 *     SII_S += val prod_{i in S} (o_i - z_i) int_0^1 prod_{j not in S} a_j(p) dp,
 * integrated with n_quad Gauss-Legendre points (exact when the path has at most
 * 2 n_quad + s - 1 unique features, Thm 2).  Output, compact:
 *   out    device, M x C(F, s) fp32, overwritten; entry [sample][rank] for the
 *          features a_1 < ... < a_s, rank = their lexicographic rank among the
 *          C(F, s) subsets (s = 3 gives the layout of qts_shap_interactions3)
 * Cross-path accumulation is FP64 in the ensemble's workspace (C(F, s) * M
 * doubles, grown on demand with cudaMalloc).  Paths of at most 16 unique
 * features, FP32 tables only; QTS_ERR_ARG for s outside [2, 8],
 * QTS_ERR_UNSUPPORTED beyond those limits or when C(F, s) * M > 2^40.
 */
qts_status qts_shap_interactions_order(qts_ensemble *ens, const float *X, int64_t M, int32_t F,
                                       int32_t order, int32_t n_quad, float *out, qts_stream_t stream);

/*
 * qts_shap_interactions_noalloc - qts_shap_interactions without any device
 * allocation.  No counterpart in the paper: this is for callers that must not
 * allocate device memory during the call - code running while a CUDA stream is
 * being captured into a graph that forbids allocation nodes, services with a
 * fixed memory budget whose allocator owns all device memory, or latency-bound
 * callers that cannot afford cudaMalloc's implicit device synchronisation.
 * The FP64 accumulators live in ONE fixed array compiled into the library
 * (16 MiB on every device that loads it, held until the process exits), so the
 * call supports (F(F-1)/2 + F) * M <= 2,097,152 and returns QTS_ERR_UNSUPPORTED,
 * with a message, beyond that.  The first call on a device (and the first after
 * a reset of that device) looks the array's address up with
 * cudaGetSymbolAddress; make that first call before any stream capture.  Every
 * call clears the part of the array it uses and reuses it, and there is one
 * array per device for the whole process - shared by every ensemble and every
 * handle - so calls that overlap on the GPU (different streams, threads or
 * ensembles) race and give wrong results: serialise all calls on a device
 * across the process, not per ensemble.  Arguments and output layout as
 * qts_shap_interactions; it runs on the per-leaf path tables (building the
 * sibling-pair tables would allocate), so its sums match
 * qts_shap_interactions' to rounding, not bit for bit.
 */
qts_status qts_shap_interactions_noalloc(qts_ensemble *ens, const float *X, int64_t M, int32_t F,
                                         int32_t n_quad, float *phi_ij, qts_stream_t stream);

/*
 * qts_shap_backward - adjoint of qts_shap_values.  With
 * L = sum_s sum_{f <= F} grad_phi[s][f] * phi[s][f]:
 *   d_leaf  device, N fp64 (N = total nodes), overwritten: dL/d leaf_value[n]
 *           (0 at internal nodes)
 *   d_z     device, N fp64, overwritten: dL/d z[n] (0 at roots)
 * The paper has no adjoint; this differentiates Thm 1 / Eq.
 * shap_as_weighted_banzhafs with the same n_quad rule, recomputing per-path
 * products instead of storing them.
 *   grad_phi device, M x (F+1) fp32 (column F weights the bias E[f]).
 * FP32 ensembles run on the sibling-pair tables (built on first use, as for
 * qts_shap_values); a pair's dL/dval is split over its two leaves exactly.
 */
qts_status qts_shap_backward(qts_ensemble *ens, const float *X, int64_t M, int32_t F,
                             int32_t n_quad, const float *grad_phi, double *d_leaf, double *d_z,
                             qts_stream_t stream);

/* One request of a batched call; all pointers are device pointers. */
typedef struct qts_request {
    qts_ensemble *ens;
    const float *X;        /* M x F */
    int64_t M;
    int32_t F;
    const float *grad_phi; /* M x (F+1); NULL = forward only */
    double *phi;           /* M x (F+1), overwritten (may be NULL when grad_phi != NULL) */
    double *d_leaf;        /* N, overwritten (ignored when grad_phi == NULL) */
    double *d_z;           /* N, overwritten (ignored when grad_phi == NULL) */
} qts_request;

/*
 * qts_batched_fwd_bwd - forward (and, where grad_phi is given, backward) of many
 * heterogeneous requests in ONE persistent kernel launch: a device work list of
 * (request, path bucket, path chunk, sample tile) items sorted by cost is
 * consumed through an atomic counter, and one pass over each (sample, path)
 * produces both phi and the adjoint (the forward product terms are a subset of
 * the adjoint's).  The whole call (initialisation, persistent kernel, adjoint
 * epilogue) is captured once into a CUDA graph keyed by the request set and
 * replayed on later calls with the same requests.  Each ensemble may appear in
 * at most one request of a call.  FP32 ensembles only.  n_quad as
 * qts_shap_values; with QTS_NQ_EXACT every bucket takes ceil(D / 2) points for
 * its width D and the graph holds one persistent launch per (register class,
 * accumulator-tile size, rule).
 */
qts_status qts_batched_fwd_bwd(int32_t n_requests, const qts_request *reqs, int32_t n_quad,
                               qts_stream_t stream);

/*
 * qts_batched_autotune - pick the batched launch's per-width parameters for a
 * set of requests by timing its persistent kernel on the requests' own data (the
 * autotuner of the batched form; the paper has no batching).  For every bucket
 * width that carries at least 1% of the batch's work it times, with that
 * width's work items alone in the launch, the paths per work item (one, two,
 * four and eight times the default, at most 4,096) and, where the fused pass
 * packs two samples per lane,
 * the sample mapping (each warp its own 64 samples, or the block's warps sharing
 * 64 samples and splitting the paths), and keeps the fastest.  Then, for the
 * register classes of widths 1-6 and 7-10 (four and three blocks per SM), it
 * times the class's launch with all blocks that fit and with one fewer, which
 * leaves more of the SM's shared memory to L1, and keeps the faster.  The
 * choices are stored in each request's ensemble and used by later batched
 * calls that include it (their cached graphs are rebuilt).
 *   reqs, n, n_quad  as qts_batched_fwd_bwd; the requests' outputs are
 *                    overwritten with partial results
 *   max_samples      time on the first min(M, max_samples) samples of each
 *                    request (0: all)
 *   chosen           host, 3 * (QTS_MAX_UNIQUE_FEATURES_PER_PATH + 1) int32 or
 *                    NULL: for width D, [3D] paths per item, [3D + 1] mapping
 *                    (2 or 3, 0 where not packed), [3D + 2] blocks per SM of
 *                    its class (0: all that fit); 0 for untuned widths
 * Synchronous on `stream`.  Errors as qts_batched_fwd_bwd.
 */
qts_status qts_batched_autotune(int32_t n_requests, const qts_request *reqs, int32_t n_quad,
                                int64_t max_samples, int32_t *chosen, qts_stream_t stream);

/*
 * qts_get_batch_info - size of the path tables the batched pass uses for this
 * ensemble (built on first use, as by a batched call).  These tables hold each
 * pair of sibling leaves of a numerical split as one path: the pair's combined
 * leaf polynomial val_A a_A(p) + val_B a_B(p) is linear in p, so it is one more
 * element of the shared path (exact algebra of Eq. shap_as_weighted_banzhafs;
 * the paper evaluates the two paths separately).
 *   n_paths       paths, pairs counted once
 *   sum_unique    sum over paths of their unique features (the work unit)
 *   n_pair_paths  paths that stand for two leaves
 *   n_buckets     number of path-width buckets (at most 32)
 *   bucket_width, bucket_paths  host, 32 entries each: width and path count of
 *                 each bucket (entries past n_buckets are left as they are)
 * Any output pointer may be NULL.
 */
qts_status qts_get_batch_info(qts_ensemble *ens, int64_t *n_paths, int64_t *sum_unique, int64_t *n_pair_paths,
                              int32_t *n_buckets, int32_t *bucket_width, int64_t *bucket_paths);

/* Number of kernels in the graph of the calling thread's last batched call. */
int32_t qts_batched_kernel_count(void);

/* Device time (ms) of the persistent kernel(s) of the calling thread's last
 * batched call, from CUDA events recorded inside its graph (waits for them). */
qts_status qts_batched_last_kernel_ms(float *ms);

/*
 * qts_autotune - time candidate launch configurations (warps per block, paths
 * per chunk, node-group width) for this ensemble and sample count on `stream`,
 * keep the fastest in the ensemble, and, if cache_path is not NULL, merge the
 * result into that JSON file keyed by (bucket width, F range, M range).
 * X: device M x F.  Synchronous.  Scratch output is allocated internally.
 */
qts_status qts_autotune(qts_ensemble *ens, const float *X, int64_t M, int32_t F,
                        const char *cache_path, qts_stream_t stream);

/* Read and clear the ensemble's device status word after synchronising `stream`. */
qts_status qts_sync_status(qts_ensemble *ens, qts_stream_t stream);

/* Summary of the prepared path tables. */
typedef struct qts_info {
    int32_t n_trees, n_features;
    int64_t n_nodes, n_leaves, n_paths;   /* paths with >= 1 unique feature */
    int32_t max_unique;                   /* d = max unique features on a path */
    int64_t sum_unique;                   /* sum over paths of unique features */
    int32_t n_buckets;
    int32_t bucket_width[32];
    int64_t bucket_paths[32];
    double expected_value;                /* E[f] */
    int64_t device_bytes;                 /* path tables + adjoint metadata */
    uint32_t flags;
} qts_info;
qts_status qts_get_info(const qts_ensemble *ens, qts_info *out);

/*
 * qts_describe_ensemble - host-only dry run of qts_load_ensemble's path
 * preparation (Sec. 2 merging and bucketing): same arguments and checks, no
 * device memory is touched; fills `out` (device_bytes = the bytes an upload
 * would take).  Usable without a GPU.  With QTS_DESCRIBE_PAIRS in flags it
 * describes the tables of the batched pass instead (sibling leaves of a
 * numerical split as one path; see qts_get_batch_info).
 */
#define QTS_DESCRIBE_PAIRS 2u
qts_status qts_describe_ensemble(int32_t n_trees, const int64_t *tree_node_offsets,
                                 const int32_t *left, const int32_t *right, const int32_t *feature,
                                 const float *threshold, const uint8_t *default_left,
                                 const float *z, const float *leaf_value, int32_t n_features,
                                 uint32_t flags, qts_info *out);

/*
 * qts_selftest_wait_timeout - exercise the device failure path (no counterpart
 * in the paper).  Enqueues one block on `stream` that waits, with the same
 * bounded wait the kernels use for their bulk copies, on a barrier that nothing
 * completes; after about a second the wait gives up and latches
 * QTS_ERR_TIMEOUT in the ensemble's status word, which the next
 * qts_sync_status returns (and clears).  The context stays usable.
 */
qts_status qts_selftest_wait_timeout(qts_ensemble *ens, qts_stream_t stream);

/*
 * qts_describe_paths - host-only: the FP32 path tables that
 * qts_load_ensemble_cat would upload (Sec. 2: paths merged per feature,
 * Eq. q_def; bucketed by width), for inspection and tests.  No device memory is
 * touched.  Call once with records == NULL to get *n_records and *n_paths, then
 * again with buffers of those sizes.
 *   records     host, n_records x 4 uint32: each path of a bucket of width D is
 *               D + 1 records, the header {val, prod z, 0, 0} and the elements
 *               {z, lo, hi, bits} sorted by feature (floats as IEEE-754 bit
 *               patterns); bits = feature | 0x80000000 (NaN satisfies every
 *               merged split) | 0x40000000 (categorical: lo and hi hold the low
 *               and high 32 bits of the merged category set) | 0x20000000
 *               (values that are no category satisfy it); padding elements are
 *               {1, -inf, +inf, n_features | 0x80000000}
 *   path_leaf   host, n_paths: global node index of each path's leaf
 *   path_width  host, n_paths: the width D of each path's bucket
 * Buckets come in increasing width, the paths of a bucket in tree order and,
 * within a tree, left subtree first.  Other arguments as
 * qts_load_ensemble_cat (is_categorical may be NULL).  Errors as
 * qts_load_ensemble_cat, plus QTS_ERR_ARG when a buffer is NULL on the second
 * call.
 */
qts_status qts_describe_paths(int32_t n_trees, const int64_t *tree_node_offsets, const int32_t *left,
                              const int32_t *right, const int32_t *feature, const float *threshold,
                              const uint8_t *default_left, const float *z, const float *leaf_value,
                              const uint8_t *is_categorical, const uint64_t *category_left_mask,
                              int32_t n_features, int64_t *n_records, int64_t *n_paths,
                              uint32_t *records, int64_t *path_leaf, int32_t *path_width);

/*
 * qts_describe_alg1_program - host-only: the record program that
 * qts_shap_values_alg1 walks (Algorithm 1, Sec. 5), for inspection and tests.
 * No device memory is touched.  Call once with records == NULL to get
 * *n_records, then again with buffers.
 *   records   host, n_records x 8 uint32: one record per internal node, each
 *             tree's nodes in preorder (a node, then its left subtree, then its
 *             right subtree): {threshold, zc_left, zc_right, z_before, val_left,
 *             val_right, meta, depth} (floats as IEEE-754 bit patterns).
 *             zc_c = the product of the edge weights on the node's feature from
 *             the root down to and including the edge into child c; z_before =
 *             the same product above the node (1 when the feature is new on the
 *             path); val_c = child c's leaf value, 0 for an internal child;
 *             meta = feature | (depth of the nearest ancestor splitting on the
 *             same feature, 127 if none) << 16 | (child 0 is a leaf) << 23 |
 *             (child 1 is a leaf) << 24 | (NaN goes left) << 25; depth = the
 *             node's depth (root 0)
 *   tree_off  host, n_trees + 1: first record of each tree
 *   levels    host, 1: deepest internal node's depth + 1
 * Arguments otherwise as qts_load_ensemble.  Errors as qts_load_ensemble, plus
 * QTS_ERR_UNSUPPORTED for internal nodes more than 62 levels deep.
 */
qts_status qts_describe_alg1_program(int32_t n_trees, const int64_t *tree_node_offsets,
                                     const int32_t *left, const int32_t *right, const int32_t *feature,
                                     const float *threshold, const uint8_t *default_left, const float *z,
                                     const float *leaf_value, int32_t n_features, int64_t *n_records,
                                     uint32_t *records, int64_t *tree_off, int32_t *levels);

/* Gauss-Legendre nodes/weights on [0,1] used by the kernels (fp64, ascending). */
qts_status qts_gauss_legendre(int32_t n, double *t, double *w);

/*
 * qts_exact_nodes - the points QTS_NQ_EXACT takes for an order-`order` quantity
 * on paths with at most `width` unique features: ceil((width - order + 1) / 2),
 * at least 1 (Thm 2: the order-s integrand has degree at most d - s, and n
 * points integrate degree 2n - 1 exactly).  Returns 0 unless
 * 1 <= width <= QTS_MAX_UNIQUE_FEATURES_PER_PATH and order >= 1.
 */
int32_t qts_exact_nodes(int32_t width, int32_t order);

/*
 * qts_fp32_pipe_peak - measured FP32-pipe throughput of this device, the
 * denominator of the FP32 kernels' roofline: every thread of 8 blocks per SM
 * runs 16 independent FMA chains (packed != 0: 8 chains of f32x2 FMAs), timed
 * with CUDA events (fastest of three launches after one warm-up, about 20 ms
 * each).  lane_ops_per_s: FMAs per second, one per FP32 lane (an f32x2 FMA
 * counts two).  Synchronous on `stream`.  QTS_ERR_ARG for a NULL output,
 * QTS_ERR_CUDA if a launch fails.
 */
qts_status qts_fp32_pipe_peak(int32_t packed, double *lane_ops_per_s, qts_stream_t stream);

/* Thread-local description of the last error (never NULL). */
const char *qts_last_error(void);

/* Free the handle and its device memory (synchronises the device first). NULL is a no-op. */
void qts_free(qts_ensemble *ens);

#ifdef __cplusplus
}
#endif
#endif
