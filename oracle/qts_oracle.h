/*
 * FP64 CPU ORACLE for Path-Dependent Shapley values and pairwise Shapley
 * interaction values of tree ensembles.  TEST INFRASTRUCTURE ONLY: the tests,
 * the smoke check and the CPU-baseline leg of the benchmark call it; the
 * product path never does.  It shares no code with the CUDA library.
 *
 * Contents (paper sections and equations cited at each definition):
 *   orc_gl_nodes        Gauss-Legendre nodes/weights on [0,1] (Sec. 4, Sec. 6).
 *   orc_predict         plain tree prediction f(x) (Sec. 2).
 *   orc_shap_exact      phi_i by the exact integral of the Thm 1 polynomial
 *                       (Eq. ao_shap_is_intergral..., Beta identity, App. C).
 *   orc_sii_exact       pairwise SII_ij the same way (Thm 1 with |S|=2).
 *   orc_shap_quad       phi_i with n-point Gauss-Legendre instead of the exact
 *                       integral (Eq. shap_as_weighted_banzhafs).
 *   orc_sii3_exact      third-order SII_ijk the same way (Thm 1 with |S|=3).
 *   orc_brute_force     phi_i and SII_ij by subset enumeration of the
 *                       Path-Dependent game (Eq. path_dependent_game, App. C).
 *   orc_brute_force3    SII_ijk by subset enumeration.
 *   orc_alg1            Algorithm 1 (DFS with telescoping, orders 1, 2 and 3).
 *   orc_alg1_shap       Algorithm 1, first order, many samples on threads.
 *   orc_sii_order_exact order-s SII (any s) by the exact expansion (Thm 1).
 *   orc_brute_force_order  order-s SII by subset enumeration (App. C).
 *   orc_alg1_order      Algorithm 1 for any order s.
 *   orc_grad_exact      d(sum grad_phi*phi)/d(leaf values) and /d(edge weights),
 *                       differentiating Thm 1 analytically (no paper passage;
 *                       pinned by finite differences of the brute force).
 *
 * Parity pins live in tests/test_oracle_*.py; every function above is pinned.
 */
#ifndef QTS_ORACLE_H
#define QTS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Tree ensemble as node arrays; node indices are local to each tree, the root
 * of tree t is node_offsets[t].  left/right = -1 at leaves.  z[n] is the edge
 * weight w_e = n_child/n_parent of the edge into n (Sec. 2). */
typedef struct orc_ens {
    int32_t n_trees;
    int32_t n_features;
    const int64_t *node_offsets;
    const int32_t *left;
    const int32_t *right;
    const int32_t *feature;
    const float *threshold;
    const uint8_t *default_left;
    const float *z;
    const float *leaf_value;
    /* Categorical splits (both NULL when there are none): is_cat[n] = 1 makes
     * node n's split categorical; cat_left[n] holds the categories 0..63 that
     * go left.  x goes left iff it is not NaN, 0 <= x < 64 and bit floor(x) is
     * set; NaN takes default_left; any other value goes right. */
    const uint8_t *is_cat;
    const uint64_t *cat_left;
} orc_ens;

int orc_gl_nodes(int n, double *t, double *w);

void orc_predict(const orc_ens *e, const float *X, int64_t M, double *out);

/* phi: M x (F+1), last column E[f] = sum_v R_empty^v. */
int orc_shap_exact(const orc_ens *e, const float *X, int64_t M, int n_threads, double *phi);

/* sii: M x F x F symmetric with zero diagonal (the Shapley interaction index,
 * not halved); phi may be NULL, else filled like orc_shap_exact. */
int orc_sii_exact(const orc_ens *e, const float *X, int64_t M, int n_threads, double *sii,
                  double *phi);

/* phi with the integral replaced by n Gauss-Legendre points on [0,1]. */
int orc_shap_quad(const orc_ens *e, const float *X, int64_t M, int n, int n_threads, double *phi);

/* One sample; needs n_features <= 20.  phi: F+1, sii: F x F (may be NULL). */
int orc_brute_force(const orc_ens *e, const float *x, double *phi, double *sii);

/* Third-order SII_ijk (Thm 1 with |S| = 3) integrated exactly; sii3 is
 * M x F x F x F, symmetric, zero wherever two indices coincide. */
int orc_sii3_exact(const orc_ens *e, const float *X, int64_t M, int n_threads, double *sii3);

/* Third-order SII for one sample by subset enumeration; 3 <= F <= 16. */
int orc_brute_force3(const orc_ens *e, const float *x, double *sii3);

/* Algorithm 1 on one sample with n Gauss-Legendre points; order 1 fills phi
 * (F+1 incl. E[f]), order 2 fills sii (F x F, symmetric, zero diagonal),
 * order 3 fills F x F x F (symmetric, zero where indices coincide). */
int orc_alg1(const orc_ens *e, const float *x, int order, int n, double *out);

/* Order-s SII for any 1 <= s <= min(F, 16), compact: entry [sample][rank] with
 * rank the lexicographic rank of the sorted feature set among the C(F, s)
 * subsets.  Exact expansion (M samples), subset enumeration (one sample,
 * F <= 16) and Algorithm 1 with n points (one sample). */
int orc_sii_order_exact(const orc_ens *e, const float *X, int64_t M, int s, int n_threads, double *out);
int orc_brute_force_order(const orc_ens *e, const float *x, int s, double *out);
int orc_alg1_order(const orc_ens *e, const float *x, int s, int n, double *out);

/* Algorithm 1, first order, for M samples (phi: M x (F+1) incl. E[f]),
 * threaded over samples: the paper's CPU quadrature method as a baseline. */
int orc_alg1_shap(const orc_ens *e, const float *X, int64_t M, int n, int n_threads, double *phi);

/* L = sum_s sum_{f<=F} grad_phi[s,f] * phi[s,f].  Writes dL/d leaf_value and
 * dL/d z for every node (N = node_offsets[n_trees]).  If leaves != NULL only
 * the n_leaves listed leaves (global node indices) contribute, which gives
 * exact values at those leaves' own nodes (d_leaf[v], d_z[v]). */
int orc_grad_exact(const orc_ens *e, const float *X, int64_t M, const float *grad_phi,
                   const int64_t *leaves, int64_t n_leaves, int n_threads, double *d_leaf,
                   double *d_z);

/* Merged-path summary for tests: number of paths and max unique features. */
int orc_path_stats(const orc_ens *e, int64_t *n_paths, int32_t *max_d, int64_t *sum_d);

#ifdef __cplusplus
}
#endif
#endif
