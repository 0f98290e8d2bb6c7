/*
 * Seeded synthetic tree ensembles and sample matrices.
 *
 * This module only manufactures INPUTS: random-split regression trees grown on
 * synthetic N(0,1) training rows (node covers = rows routed), N(0,1) sample
 * matrices and the per-ensemble size draws of the heterogeneous batch.  It holds
 * none of the Shapley arithmetic; both the FP64 oracle and the CUDA library
 * consume what it writes, and neither shares any other code.
 *
 * Random numbers come from one counter-based generator (the splitmix64
 * finaliser of Steele, Lea and Flood, OOPSLA 2014, applied to seed-, stream-
 * and counter-derived words), so every tree, matrix row block and draw is
 * reproducible independently of threading.  Normals use Marsaglia's polar
 * method with a series logarithm written here, so the generated values are
 * the same on every IEEE-754 host compiled with -ffp-contract=off.
 */
#ifndef QTS_SYNTH_H
#define QTS_SYNTH_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct synth_ens {
    int32_t n_trees;
    int32_t n_features;
    int64_t n_nodes;          /* total over all trees */
    int64_t *node_offsets;    /* n_trees + 1; tree t owns nodes [off[t], off[t+1]) */
    int32_t *left;            /* local child index within the tree, -1 at leaves */
    int32_t *right;
    int32_t *feature;         /* split feature, -1 at leaves */
    float   *threshold;       /* x[f] < threshold goes left */
    uint8_t *default_left;    /* NaN goes left iff 1 */
    float   *z;               /* cover(n)/cover(parent(n)); 1 at the root */
    float   *leaf_value;      /* 0 at internal nodes */
    int32_t *cover;           /* leaf: max(rows routed, 1); internal: sum of children */
    int32_t max_depth_seen;
} synth_ens;

/* Grow n_trees random-split trees on n_train synthetic rows of n_features.
 * At each internal node the feature is uniform on [0, n_features) and the
 * threshold is the floor(u*n)-th smallest value (0-based) of that feature over
 * the n rows reaching the node (over all rows when none reach it).  A node is a
 * leaf at depth max_depth, or when it holds <= min_rows rows unless full_depth.
 * Leaf values ~ N(0, leaf_std^2).  Returns 0 on success, -1 on bad arguments,
 * -2 on allocation failure.  n_threads <= 0 means 1. */
int synth_grow(uint64_t seed, int n_trees, int max_depth, int min_rows, int full_depth,
               int n_features, int n_train, double leaf_std, int n_threads, synth_ens *out);

void synth_free(synth_ens *e);

/* n standard normals (float) for stream `stream`; block-parallel over n_threads. */
void synth_normal_f32(uint64_t seed, uint64_t stream, int64_t n, int n_threads, float *out);

/* Uniform double in (0,1) for (seed, stream, counter). */
double synth_uniform(uint64_t seed, uint64_t stream, uint64_t ctr);

/* Heterogeneous-batch draws for n_ens ensembles: trees log-uniform in
 * [trees_lo, trees_hi], depth uniform in {depth_lo..depth_hi}, features
 * log-uniform in [f_lo, f_hi], samples log-uniform in [m_lo, m_hi]. */
void synth_batch_draw(uint64_t seed, int n_ens, int trees_lo, int trees_hi, int depth_lo,
                      int depth_hi, int f_lo, int f_hi, int m_lo, int m_hi, int32_t *trees,
                      int32_t *depth, int32_t *nfeat, int32_t *nsamp);

#ifdef __cplusplus
}
#endif
#endif
