/*
 * FP64 CPU oracle for Quadrature-TreeSHAP (arXiv 2605.04497).
 *
 * TEST INFRASTRUCTURE: a plain, slow, obviously correct restatement of what the
 * method computes.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may call it.  It shares no code with the CUDA library.
 *
 * Build with -ffp-contract=off so results do not depend on FMA contraction.
 */
#include "qts_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ================================================ Gauss-Legendre (Sec. 4) */

/* n-point Gauss-Legendre rule mapped from [-1,1] to [0,1]:  t = (x+1)/2,
 * w = w_x/2 (Sec. 4: "Gauss-Legendre nodes and weights on [0,1]").  The roots
 * of P_n are found by Newton's method on the three-term recurrence
 *   (k+1) P_{k+1}(x) = (2k+1) x P_k(x) - k P_{k-1}(x),
 * with P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1), and w_x = 2/((1-x^2) P_n'(x)^2). */
int orc_gl_nodes(int n, double *t, double *w) {
    if (n < 1 || n > 256) return -1;
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * ((double)i + 0.75) / ((double)n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * x * p1 - (double)k * p0) / (double)(k + 1);
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = x; p0 = 1.0; }
            dp = (double)n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-17 && it > 3) break;
        }
        /* recompute the derivative at the final root for the weight */
        double p0 = 1.0, p1 = x;
        for (int k = 1; k < n; ++k) {
            double p2 = ((2.0 * k + 1.0) * x * p1 - (double)k * p0) / (double)(k + 1);
            p0 = p1;
            p1 = p2;
        }
        dp = (double)n * (x * p1 - p0) / (x * x - 1.0);
        double wx = 2.0 / ((1.0 - x * x) * dp * dp);
        /* x decreases with i; store ascending in t */
        t[i] = 0.5 * (x + 1.0);
        w[i] = 0.5 * wx;
    }
    /* ascending order */
    for (int i = 0; i < n / 2; ++i) {
        double a = t[i]; t[i] = t[n - 1 - i]; t[n - 1 - i] = a;
        double b = w[i]; w[i] = w[n - 1 - i]; w[n - 1 - i] = b;
    }
    if (n == 1) { t[0] = 0.5; w[0] = 1.0; }
    return 0;
}

/* ============================================ tree basics (Sec. 2) ======= */

/* Category test of a categorical split: is v one of the categories in mask? */
static int in_categories(uint64_t mask, float v) {
    if (!(v >= 0.0f && v < 64.0f)) return 0;
    return (int)((mask >> (int)v) & 1u);
}

/* Does x take the edge parent -> child?  x[f] < threshold goes left (a
 * categorical split: x[f]'s category is in the left set); a missing (NaN)
 * value goes the parent's default direction. */
static int takes_left(const orc_ens *e, int64_t gnode, const float *x) {
    float v = x[e->feature[gnode]];
    if (isnan(v)) return e->default_left[gnode] != 0;
    if (e->is_cat && e->is_cat[gnode]) return in_categories(e->cat_left[gnode], v);
    return v < e->threshold[gnode];
}

void orc_predict(const orc_ens *e, const float *X, int64_t M, double *out) {
    int F = e->n_features;
    for (int64_t s = 0; s < M; ++s) {
        const float *x = X + s * F;
        double acc = 0.0;
        for (int t = 0; t < e->n_trees; ++t) {
            int64_t base = e->node_offsets[t];
            int32_t v = 0;
            while (e->left[base + v] >= 0)
                v = takes_left(e, base + v, x) ? e->left[base + v] : e->right[base + v];
            acc += (double)e->leaf_value[base + v];
        }
        out[s] = acc;
    }
}

/* ==================================================== merged paths ======= */

/* One element of a root-to-leaf path after merging every split on the same
 * feature (Eq. q_def: q_i depends on "all splits on i"):
 *   z      = product of the edge weights w_e of edges on this feature
 *   [lo,hi) interval of x[f] values that satisfy all those splits
 *   nan_ok a missing x[f] satisfies them all (every split's default direction
 *          is the direction the path takes). */
typedef struct {
    int32_t feat;
    int32_t nan_ok;
    double z, lo, hi;
    /* categorical splits merged in: x[f]'s category must be in `cats`; a value
     * that is no category (outside [0, 64)) satisfies them only if other_ok */
    int32_t has_cat, other_ok;
    uint64_t cats;
    int64_t edge_begin, edge_end; /* into paths.edge_node */
} pelem;

typedef struct {
    int32_t tree;
    int32_t d;
    int64_t leaf;     /* global node index */
    double val;
    int64_t el_begin; /* into paths.el */
} ppath;

typedef struct {
    int64_t n_paths, n_el, n_edges;
    ppath *p;
    pelem *el;
    int64_t *edge_node; /* global index of the child node of each merged edge */
    int32_t max_d;
} paths_t;

typedef struct {
    int32_t feat;
    int32_t went_left;
    float thr;
    uint8_t def_left;
    uint8_t is_cat;
    uint64_t cat_left;
    double w;
    int64_t child; /* global node index */
} split_rec;

static int paths_push(paths_t *P, int64_t *cap_p, int64_t *cap_e, int64_t *cap_g, int tree,
                      int64_t leaf, double val, const split_rec *st, int depth) {
    /* distinct features in order of first appearance */
    int32_t feats[256];
    int d = 0;
    for (int k = 0; k < depth; ++k) {
        int seen = 0;
        for (int j = 0; j < d; ++j) seen |= feats[j] == st[k].feat;
        if (!seen) feats[d++] = st[k].feat;
    }
    if (P->n_paths == *cap_p) {
        *cap_p = *cap_p ? 2 * *cap_p : 1024;
        ppath *np = (ppath *)realloc(P->p, sizeof(ppath) * (size_t)*cap_p);
        if (!np) return -1;
        P->p = np;
    }
    while (P->n_el + d > *cap_e) {
        *cap_e = *cap_e ? 2 * *cap_e : 4096;
        pelem *ne = (pelem *)realloc(P->el, sizeof(pelem) * (size_t)*cap_e);
        if (!ne) return -1;
        P->el = ne;
    }
    while (P->n_edges + depth > *cap_g) {
        *cap_g = *cap_g ? 2 * *cap_g : 4096;
        int64_t *ng = (int64_t *)realloc(P->edge_node, sizeof(int64_t) * (size_t)*cap_g);
        if (!ng) return -1;
        P->edge_node = ng;
    }
    ppath *pp = &P->p[P->n_paths++];
    pp->tree = tree;
    pp->d = d;
    pp->leaf = leaf;
    pp->val = val;
    pp->el_begin = P->n_el;
    for (int j = 0; j < d; ++j) {
        pelem *el = &P->el[P->n_el++];
        el->feat = feats[j];
        el->nan_ok = 1;
        el->z = 1.0;
        el->lo = -INFINITY;
        el->hi = INFINITY;
        el->has_cat = 0;
        el->other_ok = 1;
        el->cats = ~(uint64_t)0;
        el->edge_begin = P->n_edges;
        for (int k = 0; k < depth; ++k) {
            if (st[k].feat != feats[j]) continue;
            el->z *= st[k].w;
            if (st[k].is_cat) {
                /* left: the split's categories; right: all the others, and
                 * every value that is no category */
                el->has_cat = 1;
                if (st[k].went_left) {
                    el->cats &= st[k].cat_left;
                    el->other_ok = 0;
                } else {
                    el->cats &= ~st[k].cat_left;
                }
            } else if (st[k].went_left) {
                if ((double)st[k].thr < el->hi) el->hi = (double)st[k].thr;
            } else {
                if ((double)st[k].thr > el->lo) el->lo = (double)st[k].thr;
            }
            if ((st[k].went_left != 0) != (st[k].def_left != 0)) el->nan_ok = 0;
            P->edge_node[P->n_edges++] = st[k].child;
        }
        el->edge_end = P->n_edges;
    }
    if (d > P->max_d) P->max_d = d;
    return 0;
}

typedef struct {
    const orc_ens *e;
    paths_t *P;
    int64_t cap_p, cap_e, cap_g;
    split_rec st[256];
    int tree;
    int status;
} walk_ctx;

/* Depth-first walk of one tree; st[0..depth) records the edges above v. */
static void walk(walk_ctx *W, int64_t base, int32_t v, int depth) {
    const orc_ens *e = W->e;
    int64_t g = base + v;
    if (W->status) return;
    if (e->left[g] < 0) {
        if (paths_push(W->P, &W->cap_p, &W->cap_e, &W->cap_g, W->tree, g,
                       (double)e->leaf_value[g], W->st, depth))
            W->status = -1;
        return;
    }
    if (depth >= 255) { W->status = -2; return; }
    for (int side = 0; side < 2; ++side) {
        int32_t c = side == 0 ? e->left[g] : e->right[g];
        split_rec *r = &W->st[depth];
        r->feat = e->feature[g];
        r->went_left = side == 0;
        r->thr = e->threshold[g];
        r->def_left = e->default_left[g];
        r->is_cat = (e->is_cat && e->is_cat[g]) ? 1 : 0;
        r->cat_left = r->is_cat ? e->cat_left[g] : 0;
        r->w = (double)e->z[base + c];
        r->child = base + c;
        walk(W, base, c, depth + 1);
    }
}

static int build_paths(const orc_ens *e, paths_t *P) {
    memset(P, 0, sizeof(*P));
    walk_ctx *W = (walk_ctx *)calloc(1, sizeof(walk_ctx));
    if (!W) return -1;
    W->e = e;
    W->P = P;
    for (int t = 0; t < e->n_trees && !W->status; ++t) {
        W->tree = t;
        walk(W, e->node_offsets[t], 0, 0);
    }
    int st = W->status;
    free(W);
    return st;
}

static void free_paths(paths_t *P) {
    free(P->p);
    free(P->el);
    free(P->edge_node);
    memset(P, 0, sizeof(*P));
}

/* o_j(x): 1 if x satisfies every split merged into the element, else 0. */
static double satisfied(const pelem *el, const float *x) {
    float v = x[el->feat];
    if (isnan(v)) return el->nan_ok ? 1.0 : 0.0;
    double xv = (double)v;
    int ok = el->lo <= xv && xv < el->hi;
    if (el->has_cat) {
        int in_range = v >= 0.0f && v < 64.0f;
        ok = ok && (in_range ? in_categories(el->cats, v) : el->other_ok);
    }
    return ok ? 1.0 : 0.0;
}

int orc_path_stats(const orc_ens *e, int64_t *n_paths, int32_t *max_d, int64_t *sum_d) {
    paths_t P;
    if (build_paths(e, &P)) return -1;
    *n_paths = P.n_paths;
    *max_d = P.max_d;
    *sum_d = P.n_el;
    free_paths(&P);
    return 0;
}

/* ============================== exact integral of the leaf polynomial ==== */

/* Beta identity (App. C, Lemma "Beta-function identity"):
 *   int_0^1 p^k (1-p)^(n-k) dp = k! (n-k)! / (n+1)!
 * beta[k] for k = 0..n, built from beta[0] = 1/(n+1) and
 * beta[k] = beta[k-1] * k / (n-k+1). */
static void beta_table(int n, double *beta) {
    beta[0] = 1.0 / (double)(n + 1);
    for (int k = 1; k <= n; ++k) beta[k] = beta[k - 1] * (double)k / (double)(n - k + 1);
}

/* int_0^1 prod_{j<n} ((1-p) zz[j] + p oo[j]) dp, exactly.
 * The product is expanded in the Bernstein basis p^k (1-p)^(n-k): multiplying
 * by one factor (1-p) z + p o maps coefficients c_k -> z c_k + o c_{k-1}.
 * All coefficients are >= 0, so nothing cancels.  Then each basis polynomial
 * integrates by the Beta identity.  scratch needs 2(n+1) doubles. */
static double bernstein_integral(const double *zz, const double *oo, int n, double *scratch) {
    double *c = scratch, *beta = scratch + (n + 1);
    c[0] = 1.0;
    for (int j = 0; j < n; ++j) {
        c[j + 1] = oo[j] * c[j];
        for (int k = j; k >= 1; --k) c[k] = zz[j] * c[k] + oo[j] * c[k - 1];
        c[0] = zz[j] * c[0];
    }
    beta_table(n, beta);
    double s = 0.0;
    for (int k = 0; k <= n; ++k) s += c[k] * beta[k];
    return s;
}

/* ================================================= threaded sample loop == */

typedef struct job_s {
    const orc_ens *e;
    const paths_t *P;
    const float *X;
    int64_t s_begin, s_end;
    int F;
    int n;            /* quadrature points (orc_shap_quad) */
    const double *t, *w;
    double *phi;      /* M x (F+1) */
    double *sii;      /* M x F x F */
    double bias;
} job_t;

static int run_threads(void *(*fn)(void *), job_t *proto, int64_t M, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > M) n_threads = (int)(M > 0 ? M : 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * (size_t)n_threads);
    if (!th || !jobs) { free(th); free(jobs); return -1; }
    int64_t per = (M + n_threads - 1) / n_threads;
    for (int i = 0; i < n_threads; ++i) {
        jobs[i] = *proto;
        jobs[i].s_begin = i * per < M ? i * per : M;
        jobs[i].s_end = (i + 1) * per < M ? (i + 1) * per : M;
        pthread_create(&th[i], NULL, fn, &jobs[i]);
    }
    for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    free(th);
    free(jobs);
    return 0;
}

/* E[f] = f(empty set) = sum_v R_empty^v = sum_v val(v) prod_{e in path(v)} w_e
 * (Eq. R_empty).  After merging, prod of all w_e = prod_j z_j. */
static double expected_value(const paths_t *P) {
    double b = 0.0;
    for (int64_t p = 0; p < P->n_paths; ++p) {
        double r = P->p[p].val;
        for (int j = 0; j < P->p[p].d; ++j) r *= P->el[P->p[p].el_begin + j].z;
        b += r;
    }
    return b;
}

/* --------------------------------------------------------- first order -- */

/* Thm 1 with S = {i} and Eq. R_empty: with a_j(p) = (1-p) z_j + p o_j one has
 *   R_empty (q_i - 1) prod_{j != i} (1 + (q_j - 1) p) = val (o_i - z_i) prod_{j != i} a_j(p)
 * because z_j (1 + (q_j - 1) p) = (1-p) z_j + p o_j when q_j = o_j / z_j.
 * phi_i = int_0^1 of that (Eq. ao_shap_is_intergral_of_ao_banzhaf, Cor. 1). */
static void *shap_exact_worker(void *arg) {
    job_t *J = (job_t *)arg;
    const paths_t *P = J->P;
    int F = J->F;
    int dmax = P->max_d > 0 ? P->max_d : 1;
    double *o = (double *)malloc(sizeof(double) * dmax);
    double *zz = (double *)malloc(sizeof(double) * dmax);
    double *oo = (double *)malloc(sizeof(double) * dmax);
    double *scr = (double *)malloc(sizeof(double) * 2 * (dmax + 1));
    for (int64_t s = J->s_begin; s < J->s_end; ++s) {
        const float *x = J->X + s * F;
        double *phi = J->phi + s * (F + 1);
        for (int f = 0; f <= F; ++f) phi[f] = 0.0;
        for (int64_t p = 0; p < P->n_paths; ++p) {
            const ppath *pp = &P->p[p];
            const pelem *el = P->el + pp->el_begin;
            int d = pp->d;
            for (int j = 0; j < d; ++j) o[j] = satisfied(&el[j], x);
            for (int i = 0; i < d; ++i) {
                int n = 0;
                for (int j = 0; j < d; ++j) {
                    if (j == i) continue;
                    zz[n] = el[j].z;
                    oo[n] = o[j];
                    ++n;
                }
                double I = bernstein_integral(zz, oo, n, scr);
                phi[el[i].feat] += pp->val * (o[i] - el[i].z) * I;
            }
        }
        phi[F] = J->bias;
    }
    free(o); free(zz); free(oo); free(scr);
    return NULL;
}

int orc_shap_exact(const orc_ens *e, const float *X, int64_t M, int n_threads, double *phi) {
    paths_t P;
    if (build_paths(e, &P)) return -1;
    job_t proto;
    memset(&proto, 0, sizeof(proto));
    proto.e = e; proto.P = &P; proto.X = X; proto.F = e->n_features; proto.phi = phi;
    proto.bias = expected_value(&P);
    int rc = run_threads(shap_exact_worker, &proto, M, n_threads);
    free_paths(&P);
    return rc;
}

/* --------------------------------------------------- pairwise (|S| = 2) -- */

/* Thm 1 with S = {i, j}:  SII_ij = int_0^1 val (o_i - z_i)(o_j - z_j)
 * prod_{k not in {i,j}} a_k(p) dp; leaves whose path lacks i or j add 0. */
static void *sii_exact_worker(void *arg) {
    job_t *J = (job_t *)arg;
    const paths_t *P = J->P;
    int F = J->F;
    int dmax = P->max_d > 0 ? P->max_d : 1;
    double *o = (double *)malloc(sizeof(double) * dmax);
    double *zz = (double *)malloc(sizeof(double) * dmax);
    double *oo = (double *)malloc(sizeof(double) * dmax);
    double *scr = (double *)malloc(sizeof(double) * 2 * (dmax + 1));
    for (int64_t s = J->s_begin; s < J->s_end; ++s) {
        const float *x = J->X + s * F;
        double *sii = J->sii + s * (int64_t)F * F;
        for (int64_t k = 0; k < (int64_t)F * F; ++k) sii[k] = 0.0;
        for (int64_t p = 0; p < P->n_paths; ++p) {
            const ppath *pp = &P->p[p];
            const pelem *el = P->el + pp->el_begin;
            int d = pp->d;
            for (int j = 0; j < d; ++j) o[j] = satisfied(&el[j], x);
            for (int i = 0; i < d; ++i) {
                for (int j = i + 1; j < d; ++j) {
                    int n = 0;
                    for (int k = 0; k < d; ++k) {
                        if (k == i || k == j) continue;
                        zz[n] = el[k].z;
                        oo[n] = o[k];
                        ++n;
                    }
                    double I = bernstein_integral(zz, oo, n, scr);
                    double v = pp->val * (o[i] - el[i].z) * (o[j] - el[j].z) * I;
                    sii[el[i].feat * F + el[j].feat] += v;
                    sii[el[j].feat * F + el[i].feat] += v;
                }
            }
        }
    }
    free(o); free(zz); free(oo); free(scr);
    return NULL;
}

int orc_sii_exact(const orc_ens *e, const float *X, int64_t M, int n_threads, double *sii,
                  double *phi) {
    paths_t P;
    if (build_paths(e, &P)) return -1;
    job_t proto;
    memset(&proto, 0, sizeof(proto));
    proto.e = e; proto.P = &P; proto.X = X; proto.F = e->n_features; proto.sii = sii;
    int rc = run_threads(sii_exact_worker, &proto, M, n_threads);
    if (!rc && phi) {
        proto.phi = phi;
        proto.bias = expected_value(&P);
        rc = run_threads(shap_exact_worker, &proto, M, n_threads);
    }
    free_paths(&P);
    return rc;
}

/* ----------------------------------------- n-point quadrature, 1st order -- */

/* Eq. shap_as_weighted_banzhafs: the integral replaced by sum_m w_m B_{t_m}. */
static void *shap_quad_worker(void *arg) {
    job_t *J = (job_t *)arg;
    const paths_t *P = J->P;
    int F = J->F;
    int dmax = P->max_d > 0 ? P->max_d : 1;
    double *o = (double *)malloc(sizeof(double) * dmax);
    for (int64_t s = J->s_begin; s < J->s_end; ++s) {
        const float *x = J->X + s * F;
        double *phi = J->phi + s * (F + 1);
        for (int f = 0; f <= F; ++f) phi[f] = 0.0;
        for (int64_t p = 0; p < P->n_paths; ++p) {
            const ppath *pp = &P->p[p];
            const pelem *el = P->el + pp->el_begin;
            int d = pp->d;
            for (int j = 0; j < d; ++j) o[j] = satisfied(&el[j], x);
            for (int i = 0; i < d; ++i) {
                double q = 0.0;
                for (int m = 0; m < J->n; ++m) {
                    double prod = 1.0;
                    for (int j = 0; j < d; ++j)
                        if (j != i) prod *= (1.0 - J->t[m]) * el[j].z + J->t[m] * o[j];
                    q += J->w[m] * prod;
                }
                phi[el[i].feat] += pp->val * (o[i] - el[i].z) * q;
            }
        }
        phi[F] = J->bias;
    }
    free(o);
    return NULL;
}

int orc_shap_quad(const orc_ens *e, const float *X, int64_t M, int n, int n_threads, double *phi) {
    double t[256], w[256];
    if (orc_gl_nodes(n, t, w)) return -1;
    paths_t P;
    if (build_paths(e, &P)) return -1;
    job_t proto;
    memset(&proto, 0, sizeof(proto));
    proto.e = e; proto.P = &P; proto.X = X; proto.F = e->n_features; proto.phi = phi;
    proto.n = n; proto.t = t; proto.w = w;
    proto.bias = expected_value(&P);
    int rc = run_threads(shap_quad_worker, &proto, M, n_threads);
    free_paths(&P);
    return rc;
}

/* ======================================================= brute force ====== */

/* Path-Dependent game of one tree (Eq. path_dependent_game):
 *   f(S) = sum_v R_empty^v prod_{i in S} q_i^v = sum_v val(v) prod_{e in path(v)}
 *          ( f(e) in S ? [x takes e] : w_e ),
 * evaluated top-down: a split on a feature in S follows x; any other split
 * weights both children by their edge weights. */
static double game(const orc_ens *e, int64_t base, int32_t v, const float *x, uint32_t S) {
    int64_t g = base + v;
    if (e->left[g] < 0) return (double)e->leaf_value[g];
    int32_t l = e->left[g], r = e->right[g];
    if ((S >> e->feature[g]) & 1u) return game(e, base, takes_left(e, g, x) ? l : r, x, S);
    return (double)e->z[base + l] * game(e, base, l, x, S) +
           (double)e->z[base + r] * game(e, base, r, x, S);
}

/* phi_i  = sum_{S subset of [F]\{i}} |S|! (F-|S|-1)! / F! (f(S+i) - f(S))
 * SII_ij = sum_{T subset of [F]\{i,j}} |T|! (F-|T|-2)! / (F-1)! Delta_ij f(T)
 * (App. C, the Shapley interaction index with |S| = 2). */
int orc_brute_force(const orc_ens *e, const float *x, double *phi, double *sii) {
    int F = e->n_features;
    if (F < 1 || F > 20) return -1;
    uint32_t NS = 1u << F;
    double *fs = (double *)malloc(sizeof(double) * NS);
    if (!fs) return -1;
    for (uint32_t S = 0; S < NS; ++S) {
        double acc = 0.0;
        for (int t = 0; t < e->n_trees; ++t) acc += game(e, e->node_offsets[t], 0, x, S);
        fs[S] = acc;
    }
    double fact[32];
    fact[0] = 1.0;
    for (int k = 1; k < 32; ++k) fact[k] = fact[k - 1] * (double)k;
    for (int i = 0; i < F; ++i) {
        double acc = 0.0;
        for (uint32_t S = 0; S < NS; ++S) {
            if ((S >> i) & 1u) continue;
            int k = __builtin_popcount(S);
            acc += fact[k] * fact[F - k - 1] / fact[F] * (fs[S | (1u << i)] - fs[S]);
        }
        phi[i] = acc;
    }
    phi[F] = fs[0];
    if (sii) {
        for (int i = 0; i < F; ++i) {
            sii[i * F + i] = 0.0;
            for (int j = i + 1; j < F; ++j) {
                double acc = 0.0;
                uint32_t mi = 1u << i, mj = 1u << j;
                for (uint32_t T = 0; T < NS; ++T) {
                    if (T & (mi | mj)) continue;
                    int k = __builtin_popcount(T);
                    double delta = fs[T | mi | mj] - fs[T | mi] - fs[T | mj] + fs[T];
                    acc += fact[k] * fact[F - k - 2] / fact[F - 1] * delta;
                }
                sii[i * F + j] = acc;
                sii[j * F + i] = acc;
            }
        }
    }
    free(fs);
    return 0;
}

/* ======================================================= Algorithm 1 ===== */

/* The DFS of Algorithm 1: for each (tree, sample) propagate the vector c of the
 * leaf polynomial's values at the quadrature nodes; at each edge multiply in
 * (1 + alpha_e t) and divide out the factor of the nearest ancestor edge on the
 * same feature; child subtrees return H_u = sum of their leaves' c*val*w_prod;
 * each edge adds sum_m w_m H_u delta_e gamma_P to Phi (Eq.
 * our_telescoping_background).  epsilon = 0: a seen factor is always divided
 * out unless it is exactly 1. */
typedef struct {
    const orc_ens *e;
    int64_t base;
    const float *x;
    int order, n, F;
    double t[256], w[256];
    double *p;   /* live multiplier per feature */
    int *seen;   /* p[f] != UNSEEN, equivalently f in the active set A */
    double *out; /* order 1: phi[F]; order 2: sii[F*F]; order 3: F^3; compact: C(F, s) */
    int compact; /* out is indexed by the lexicographic rank of the sorted s-subset */
} alg1_ctx;

/* C(n, k) as an exact integer (0 outside 0 <= k <= n). */
static int64_t n_choose_k(int n, int k) {
    if (k < 0 || n < k) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* Lexicographic rank of the sorted subset c[0] < ... < c[s-1] of {0..F-1}:
 * the subsets before it are those that agree on c[0..i-1] and have a smaller
 * i-th element, counted position by position. */
static int64_t subset_rank(const int *c, int s, int F) {
    int64_t r = 0;
    int prev = -1;
    for (int i = 0; i < s; ++i) {
        r += n_choose_k(F - prev - 1, s - i) - n_choose_k(F - c[i], s - i);
        prev = c[i];
    }
    return r;
}

static void sort_ints(int *c, int s) {
    for (int i = 1; i < s; ++i) {
        int v = c[i], k = i - 1;
        while (k >= 0 && c[k] > v) { c[k + 1] = c[k]; --k; }
        c[k + 1] = v;
    }
}

/* Order-s update of one edge on feature f (Alg. 1): every (s-1)-subset P of the
 * active set without f adds sum_m w_m H_u delta_e prod_{j in P} gamma_j. */
static void alg1_subsets(alg1_ctx *C, int f, const double *Hu, const double *delta) {
    const int F = C->F, s = C->order, n = C->n;
    int act[256], na = 0;
    for (int j = 0; j < F; ++j)
        if (j != f && C->seen[j]) act[na++] = j;
    const int r = s - 1;
    if (na < r) return;
    int idx[16];
    for (int i = 0; i < r; ++i) idx[i] = i;
    for (;;) {
        double acc = 0.0;
        for (int m = 0; m < n; ++m) {
            double g = C->w[m] * Hu[m] * delta[m];
            for (int i = 0; i < r; ++i) {
                double aj = C->p[act[idx[i]]] - 1.0;
                g *= aj / (1.0 + aj * C->t[m]);
            }
            acc += g;
        }
        int c[16];
        for (int i = 0; i < r; ++i) c[i] = act[idx[i]];
        c[r] = f;
        sort_ints(c, s);
        C->out[subset_rank(c, s, F)] += acc;
        /* next (s-1)-combination of 0..na-1 */
        int i = r - 1;
        while (i >= 0 && idx[i] == na - r + i) --i;
        if (i < 0) break;
        ++idx[i];
        for (int k = i + 1; k < r; ++k) idx[k] = idx[k - 1] + 1;
    }
}

static void alg1_dfs(alg1_ctx *C, int32_t v, const double *c, double wprod, double *H) {
    const orc_ens *e = C->e;
    int n = C->n;
    int64_t g = C->base + v;
    if (e->left[g] < 0) {
        for (int m = 0; m < n; ++m) H[m] = c[m] * (double)e->leaf_value[g] * wprod;
        return;
    }
    int f = e->feature[g];
    int goes_left = takes_left(e, g, C->x);
    double cp[256], Hu[256], delta[256];
    for (int m = 0; m < n; ++m) H[m] = 0.0;
    for (int side = 0; side < 2; ++side) {
        int32_t u = side == 0 ? e->left[g] : e->right[g];
        double we = (double)e->z[C->base + u];
        int se = (side == 0) == (goes_left != 0);
        double pe, pup;
        int was_seen = C->seen[f];
        double pold = C->p[f];
        if (!was_seen) {
            pe = se ? 1.0 / we : 0.0;
            pup = 1.0;
        } else if (pold == 0.0) {
            pe = 0.0;
            pup = 0.0;
        } else {
            pe = se ? pold / we : 0.0;
            pup = pold;
        }
        double ae = pe - 1.0;
        for (int m = 0; m < n; ++m) cp[m] = c[m] * (1.0 + ae * C->t[m]);
        if (was_seen && pold != 1.0)
            for (int m = 0; m < n; ++m) cp[m] /= (1.0 + (pold - 1.0) * C->t[m]);
        C->p[f] = pe;
        C->seen[f] = 1;
        alg1_dfs(C, u, cp, wprod * we, Hu);
        double aup = pup - 1.0;
        for (int m = 0; m < n; ++m)
            delta[m] = ae / (1.0 + ae * C->t[m]) - aup / (1.0 + aup * C->t[m]);
        if (C->compact) {
            alg1_subsets(C, f, Hu, delta);
        } else if (C->order == 1) {
            double acc = 0.0;
            for (int m = 0; m < n; ++m) acc += C->w[m] * Hu[m] * delta[m];
            C->out[f] += acc;
        } else if (C->order == 2) {
            for (int j = 0; j < C->F; ++j) {
                if (j == f || !C->seen[j]) continue;
                double aj = C->p[j] - 1.0, acc = 0.0;
                for (int m = 0; m < n; ++m)
                    acc += C->w[m] * Hu[m] * delta[m] * (aj / (1.0 + aj * C->t[m]));
                C->out[j * C->F + f] += acc;
                C->out[f * C->F + j] += acc;
            }
        } else {
            /* s = 3: every 2-subset {j, k} of the active set without f */
            const int F = C->F;
            for (int j = 0; j < F; ++j) {
                if (j == f || !C->seen[j]) continue;
                for (int k = j + 1; k < F; ++k) {
                    if (k == f || !C->seen[k]) continue;
                    double aj = C->p[j] - 1.0, ak = C->p[k] - 1.0, acc = 0.0;
                    for (int m = 0; m < n; ++m)
                        acc += C->w[m] * Hu[m] * delta[m] * (aj / (1.0 + aj * C->t[m])) *
                               (ak / (1.0 + ak * C->t[m]));
                    int64_t F2 = (int64_t)F * F;
                    C->out[j * F2 + k * F + f] += acc;
                    C->out[j * F2 + f * F + k] += acc;
                    C->out[k * F2 + j * F + f] += acc;
                    C->out[k * F2 + f * F + j] += acc;
                    C->out[f * F2 + j * F + k] += acc;
                    C->out[f * F2 + k * F + j] += acc;
                }
            }
        }
        C->p[f] = pold;
        C->seen[f] = was_seen;
        for (int m = 0; m < n; ++m) H[m] += Hu[m];
    }
}

static double tree_bias(const orc_ens *e, int64_t base, int32_t v) {
    int64_t g = base + v;
    if (e->left[g] < 0) return (double)e->leaf_value[g];
    int32_t l = e->left[g], r = e->right[g];
    return (double)e->z[base + l] * tree_bias(e, base, l) + (double)e->z[base + r] * tree_bias(e, base, r);
}

int orc_alg1(const orc_ens *e, const float *x, int order, int n, double *out) {
    if (order < 1 || order > 3) return -1;
    alg1_ctx *C = (alg1_ctx *)calloc(1, sizeof(alg1_ctx));
    if (!C) return -1;
    if (orc_gl_nodes(n, C->t, C->w)) { free(C); return -1; }
    int F = e->n_features;
    C->e = e; C->x = x; C->order = order; C->n = n; C->F = F; C->out = out;
    C->p = (double *)calloc((size_t)F, sizeof(double));
    C->seen = (int *)calloc((size_t)F, sizeof(int));
    int64_t nout = order == 1 ? F + 1 : (order == 2 ? (int64_t)F * F : (int64_t)F * F * F);
    for (int64_t k = 0; k < nout; ++k) out[k] = 0.0;
    double ones[256], H[256];
    for (int m = 0; m < n; ++m) ones[m] = 1.0;
    double bias = 0.0;
    for (int t = 0; t < e->n_trees; ++t) {
        C->base = e->node_offsets[t];
        alg1_dfs(C, 0, ones, 1.0, H);
        bias += tree_bias(e, C->base, 0);
    }
    if (order == 1) out[F] = bias;
    free(C->p);
    free(C->seen);
    free(C);
    return 0;
}

/* Order-s Shapley interaction index for any s (Thm 1 with |S| = s): per
 * merged path and s-subset S of its elements,
 *   SII_S += val prod_{i in S} (o_i - z_i) int_0^1 prod_{j not in S} a_j(p) dp,
 * integrated exactly (Bernstein form).  Output compact: M x C(F, s), entry
 * [sample][rank] with rank the lexicographic rank of the sorted feature set. */
typedef struct {
    const paths_t *P;
    const float *X;
    int64_t s_begin, s_end;
    int F, s;
    int64_t n_sub;
    double *out;
} ojob_t;

static void *order_exact_worker(void *arg) {
    ojob_t *J = (ojob_t *)arg;
    const paths_t *P = J->P;
    const int F = J->F, s = J->s;
    int dmax = P->max_d > 0 ? P->max_d : 1;
    double *o = (double *)malloc(sizeof(double) * dmax);
    double *zz = (double *)malloc(sizeof(double) * dmax);
    double *oo = (double *)malloc(sizeof(double) * dmax);
    double *scr = (double *)malloc(sizeof(double) * 2 * (dmax + 1));
    int *in = (int *)malloc(sizeof(int) * dmax);
    for (int64_t sm = J->s_begin; sm < J->s_end; ++sm) {
        const float *x = J->X + sm * F;
        double *out = J->out + sm * J->n_sub;
        for (int64_t q = 0; q < J->n_sub; ++q) out[q] = 0.0;
        for (int64_t p = 0; p < P->n_paths; ++p) {
            const ppath *pp = &P->p[p];
            const pelem *el = P->el + pp->el_begin;
            const int d = pp->d;
            if (d < s) continue;
            for (int j = 0; j < d; ++j) o[j] = satisfied(&el[j], x);
            int idx[16];
            for (int i = 0; i < s; ++i) idx[i] = i;
            for (;;) {
                for (int j = 0; j < d; ++j) in[j] = 0;
                double v = pp->val;
                int c[16];
                for (int i = 0; i < s; ++i) {
                    in[idx[i]] = 1;
                    v *= o[idx[i]] - el[idx[i]].z;
                    c[i] = el[idx[i]].feat;
                }
                int n = 0;
                for (int l = 0; l < d; ++l) {
                    if (in[l]) continue;
                    zz[n] = el[l].z;
                    oo[n] = o[l];
                    ++n;
                }
                v *= bernstein_integral(zz, oo, n, scr);
                sort_ints(c, s);
                out[subset_rank(c, s, F)] += v;
                int i = s - 1;
                while (i >= 0 && idx[i] == d - s + i) --i;
                if (i < 0) break;
                ++idx[i];
                for (int k = i + 1; k < s; ++k) idx[k] = idx[k - 1] + 1;
            }
        }
    }
    free(o); free(zz); free(oo); free(scr); free(in);
    return NULL;
}

int orc_sii_order_exact(const orc_ens *e, const float *X, int64_t M, int s, int n_threads, double *out) {
    const int F = e->n_features;
    if (s < 1 || s > 16 || s > F) return -1;
    paths_t P;
    if (build_paths(e, &P)) return -1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > M) n_threads = (int)(M > 0 ? M : 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    ojob_t *jobs = (ojob_t *)malloc(sizeof(ojob_t) * (size_t)n_threads);
    if (!th || !jobs) { free(th); free(jobs); free_paths(&P); return -1; }
    int64_t per = (M + n_threads - 1) / n_threads;
    for (int i = 0; i < n_threads; ++i) {
        jobs[i].P = &P;
        jobs[i].X = X;
        jobs[i].F = F;
        jobs[i].s = s;
        jobs[i].n_sub = n_choose_k(F, s);
        jobs[i].out = out;
        jobs[i].s_begin = i * per < M ? i * per : M;
        jobs[i].s_end = (i + 1) * per < M ? (i + 1) * per : M;
        pthread_create(&th[i], NULL, order_exact_worker, &jobs[i]);
    }
    for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    free(th);
    free(jobs);
    free_paths(&P);
    return 0;
}

/* Order-s SII for one sample by subset enumeration (App. C):
 *   SII_S = sum_{T subset of [F] \ S} |T|! (F - |T| - s)! / (F - s + 1)! Delta_S f(T),
 *   Delta_S f(T) = sum_{L subset of S} (-1)^(s - |L|) f(T + L).
 * Compact output C(F, s); needs s <= F <= 16. */
int orc_brute_force_order(const orc_ens *e, const float *x, int s, double *out) {
    const int F = e->n_features;
    if (s < 1 || s > F || F > 16) return -1;
    uint32_t NS = 1u << F;
    double *fs = (double *)malloc(sizeof(double) * NS);
    if (!fs) return -1;
    for (uint32_t S = 0; S < NS; ++S) {
        double acc = 0.0;
        for (int t = 0; t < e->n_trees; ++t) acc += game(e, e->node_offsets[t], 0, x, S);
        fs[S] = acc;
    }
    double fact[40];
    fact[0] = 1.0;
    for (int k = 1; k < 40; ++k) fact[k] = fact[k - 1] * (double)k;
    int idx[16];
    for (int i = 0; i < s; ++i) idx[i] = i;
    int64_t rank = 0;
    for (;;) {
        uint32_t mS = 0;
        for (int i = 0; i < s; ++i) mS |= 1u << idx[i];
        double sii = 0.0;
        for (uint32_t T = 0; T < NS; ++T) {
            if (T & mS) continue;
            int t = __builtin_popcount(T);
            double wgt = fact[t] * fact[F - t - s] / fact[F - s + 1];
            double delta = 0.0;
            for (uint32_t L = mS;; L = (L - 1) & mS) {
                int l = __builtin_popcount(L);
                delta += ((s - l) % 2 ? -1.0 : 1.0) * fs[T | L];
                if (L == 0) break;
            }
            sii += wgt * delta;
        }
        out[rank++] = sii;  /* combinations are visited in lexicographic order */
        int i = s - 1;
        while (i >= 0 && idx[i] == F - s + i) --i;
        if (i < 0) break;
        ++idx[i];
        for (int k = i + 1; k < s; ++k) idx[k] = idx[k - 1] + 1;
    }
    free(fs);
    return 0;
}

/* Algorithm 1 for any order s on one sample with n points; compact output
 * C(F, s) in lexicographic order. */
int orc_alg1_order(const orc_ens *e, const float *x, int s, int n, double *out) {
    const int F = e->n_features;
    if (s < 1 || s > 16 || s > F) return -1;
    alg1_ctx *C = (alg1_ctx *)calloc(1, sizeof(alg1_ctx));
    if (!C) return -1;
    if (orc_gl_nodes(n, C->t, C->w)) { free(C); return -1; }
    C->e = e; C->x = x; C->order = s; C->n = n; C->F = F; C->out = out; C->compact = 1;
    C->p = (double *)calloc((size_t)F, sizeof(double));
    C->seen = (int *)calloc((size_t)F, sizeof(int));
    const int64_t nout = n_choose_k(F, s);
    for (int64_t k = 0; k < nout; ++k) out[k] = 0.0;
    double ones[256], H[256];
    for (int m = 0; m < n; ++m) ones[m] = 1.0;
    for (int t = 0; t < e->n_trees; ++t) {
        C->base = e->node_offsets[t];
        if (e->left[C->base] >= 0) alg1_dfs(C, 0, ones, 1.0, H);
    }
    free(C->p);
    free(C->seen);
    free(C);
    return 0;
}

/* Algorithm 1 as a CPU quadrature method: first-order phi for M samples with
 * n Gauss-Legendre points, threads over samples (each thread runs the DFS of
 * orc_alg1 on its rows).  This is the paper's own CPU formulation (Sec. 5,
 * Algorithm 1), not the exact expansion. */
typedef struct {
    const orc_ens *e;
    const float *X;
    int64_t s_begin, s_end;
    int n;
    double *phi;
    int rc;
} a1job_t;

static void *alg1_shap_worker(void *arg) {
    a1job_t *J = (a1job_t *)arg;
    const int F = J->e->n_features;
    for (int64_t s = J->s_begin; s < J->s_end; ++s)
        if (orc_alg1(J->e, J->X + s * F, 1, J->n, J->phi + s * (F + 1)) != 0) J->rc = -1;
    return NULL;
}

int orc_alg1_shap(const orc_ens *e, const float *X, int64_t M, int n, int n_threads, double *phi) {
    if (M < 0 || n < 1 || n > 256) return -1;
    if (M == 0) return 0;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > M) n_threads = (int)M;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    a1job_t *jobs = (a1job_t *)malloc(sizeof(a1job_t) * (size_t)n_threads);
    if (!th || !jobs) { free(th); free(jobs); return -1; }
    int64_t per = (M + n_threads - 1) / n_threads;
    for (int i = 0; i < n_threads; ++i) {
        jobs[i].e = e;
        jobs[i].X = X;
        jobs[i].n = n;
        jobs[i].phi = phi;
        jobs[i].rc = 0;
        jobs[i].s_begin = i * per < M ? i * per : M;
        jobs[i].s_end = (i + 1) * per < M ? (i + 1) * per : M;
        pthread_create(&th[i], NULL, alg1_shap_worker, &jobs[i]);
    }
    int rc = 0;
    for (int i = 0; i < n_threads; ++i) {
        pthread_join(th[i], NULL);
        if (jobs[i].rc) rc = -1;
    }
    free(th);
    free(jobs);
    return rc;
}

/* ========================================================= gradients ===== */

/* L = sum_s sum_i g_{s,f_i} phi_{s,f_i} + sum_s grad_phi[s,F] E[f], with
 * phi_i = val d_i I_i, d_i = o_i - z_i, I_i = int prod_{j != i} a_j, and
 * a_j(p) = (1-p) z_j + p o_j.  Per merged path:
 *   dL/dval = sum_s sum_i g_i d_i I_i + G prod_j z_j,            G = sum_s grad_phi[s,F]
 *   dL/dz_k = sum_s val ( -g_k I_k + sum_{i != k} g_i d_i J_ik ) + G val prod_{j != k} z_j,
 *   J_ik    = int (1-p) prod_{j not in {i,k}} a_j(p) dp   (d a_k / d z_k = 1-p).
 * (1-p) is itself a factor (1-p)*1 + p*0, so J_ik is one more Bernstein
 * integral.  Edge weights merged into element k receive
 *   dL/dw_e = dL/dz_k * prod_{e' in k, e' != e} w_e'. */
typedef struct gjob_s {
    const orc_ens *e;
    const paths_t *P;
    const float *X, *grad;
    int64_t M;
    int F;
    const int64_t *plist;
    int64_t p_begin, p_end;
    double G;
    double *dval; /* per listed path */
    double *dz;   /* per element of listed path, indexed by el index */
} gjob_t;

static void *grad_worker(void *arg) {
    gjob_t *J = (gjob_t *)arg;
    const paths_t *P = J->P;
    int F = J->F;
    int dmax = P->max_d > 0 ? P->max_d : 1;
    double *o = (double *)malloc(sizeof(double) * dmax);
    double *zz = (double *)malloc(sizeof(double) * (dmax + 1));
    double *oo = (double *)malloc(sizeof(double) * (dmax + 1));
    double *I = (double *)malloc(sizeof(double) * dmax);
    double *scr = (double *)malloc(sizeof(double) * 2 * (dmax + 2));
    for (int64_t q = J->p_begin; q < J->p_end; ++q) {
        int64_t p = J->plist[q];
        const ppath *pp = &P->p[p];
        const pelem *el = P->el + pp->el_begin;
        int d = pp->d;
        double dval = 0.0;
        double *dz = J->dz + pp->el_begin;
        for (int k = 0; k < d; ++k) dz[k] = 0.0;
        for (int64_t s = 0; s < J->M; ++s) {
            const float *x = J->X + s * F;
            const float *gr = J->grad + s * (F + 1);
            for (int j = 0; j < d; ++j) o[j] = satisfied(&el[j], x);
            for (int i = 0; i < d; ++i) {
                int n = 0;
                for (int j = 0; j < d; ++j) {
                    if (j == i) continue;
                    zz[n] = el[j].z; oo[n] = o[j]; ++n;
                }
                I[i] = bernstein_integral(zz, oo, n, scr);
                dval += (double)gr[el[i].feat] * (o[i] - el[i].z) * I[i];
            }
            for (int k = 0; k < d; ++k) {
                double acc = -(double)gr[el[k].feat] * I[k];
                for (int i = 0; i < d; ++i) {
                    if (i == k) continue;
                    int n = 0;
                    for (int j = 0; j < d; ++j) {
                        if (j == i || j == k) continue;
                        zz[n] = el[j].z; oo[n] = o[j]; ++n;
                    }
                    zz[n] = 1.0; oo[n] = 0.0; ++n; /* the factor (1-p) */
                    double Jik = bernstein_integral(zz, oo, n, scr);
                    acc += (double)gr[el[i].feat] * (o[i] - el[i].z) * Jik;
                }
                dz[k] += pp->val * acc;
            }
        }
        double zall = 1.0;
        for (int j = 0; j < d; ++j) zall *= el[j].z;
        dval += J->G * zall;
        for (int k = 0; k < d; ++k) {
            double zo = 1.0;
            for (int j = 0; j < d; ++j) if (j != k) zo *= el[j].z;
            dz[k] += J->G * pp->val * zo;
        }
        J->dval[q] = dval;
    }
    free(o); free(zz); free(oo); free(I); free(scr);
    return NULL;
}

int orc_grad_exact(const orc_ens *e, const float *X, int64_t M, const float *grad_phi,
                   const int64_t *leaves, int64_t n_leaves, int n_threads, double *d_leaf,
                   double *d_z) {
    paths_t P;
    if (build_paths(e, &P)) return -1;
    int F = e->n_features;
    int64_t N = e->node_offsets[e->n_trees];
    /* which paths contribute */
    int64_t np = 0;
    int64_t *plist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P.n_paths > 0 ? P.n_paths : 1));
    if (leaves) {
        for (int64_t q = 0; q < n_leaves; ++q)
            for (int64_t p = 0; p < P.n_paths; ++p)
                if (P.p[p].leaf == leaves[q]) { plist[np++] = p; break; }
    } else {
        for (int64_t p = 0; p < P.n_paths; ++p) plist[np++] = p;
    }
    double G = 0.0;
    for (int64_t s = 0; s < M; ++s) G += (double)grad_phi[s * (F + 1) + F];
    double *dval = (double *)calloc((size_t)(np > 0 ? np : 1), sizeof(double));
    double *dz = (double *)calloc((size_t)(P.n_el > 0 ? P.n_el : 1), sizeof(double));
    if (n_threads < 1) n_threads = 1;
    if (n_threads > np) n_threads = (int)(np > 0 ? np : 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    gjob_t *jobs = (gjob_t *)malloc(sizeof(gjob_t) * (size_t)n_threads);
    int64_t per = (np + n_threads - 1) / n_threads;
    for (int i = 0; i < n_threads; ++i) {
        jobs[i] = (gjob_t){e, &P, X, grad_phi, M, F, plist,
                           i * per < np ? i * per : np, (i + 1) * per < np ? (i + 1) * per : np,
                           G, dval, dz};
        pthread_create(&th[i], NULL, grad_worker, &jobs[i]);
    }
    for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    for (int64_t k = 0; k < N; ++k) { d_leaf[k] = 0.0; d_z[k] = 0.0; }
    /* chain rule to the edges, serially (fixed summation order) */
    for (int64_t q = 0; q < np; ++q) {
        const ppath *pp = &P.p[plist[q]];
        d_leaf[pp->leaf] += dval[q];
        for (int k = 0; k < pp->d; ++k) {
            const pelem *el = &P.el[pp->el_begin + k];
            for (int64_t a = el->edge_begin; a < el->edge_end; ++a) {
                double others = 1.0;
                for (int64_t b = el->edge_begin; b < el->edge_end; ++b)
                    if (b != a) others *= (double)e->z[P.edge_node[b]];
                d_z[P.edge_node[a]] += dz[pp->el_begin + k] * others;
            }
        }
    }
    free(th); free(jobs); free(dval); free(dz); free(plist);
    free_paths(&P);
    return 0;
}

/* ================================================== third order (|S| = 3) */

/* Thm 1 with S = {i, j, k}: SII_ijk = int_0^1 val (o_i - z_i)(o_j - z_j)(o_k - z_k)
 * prod_{l not in {i,j,k}} a_l(p) dp (Eq. ao_shap_is_intergral_of_ao_banzhaf). */
static void *sii3_exact_worker(void *arg) {
    job_t *J = (job_t *)arg;
    const paths_t *P = J->P;
    int F = J->F;
    int64_t F2 = (int64_t)F * F, F3 = F2 * F;
    int dmax = P->max_d > 0 ? P->max_d : 1;
    double *o = (double *)malloc(sizeof(double) * dmax);
    double *zz = (double *)malloc(sizeof(double) * dmax);
    double *oo = (double *)malloc(sizeof(double) * dmax);
    double *scr = (double *)malloc(sizeof(double) * 2 * (dmax + 1));
    for (int64_t s = J->s_begin; s < J->s_end; ++s) {
        const float *x = J->X + s * F;
        double *out = J->sii + s * F3;
        for (int64_t q = 0; q < F3; ++q) out[q] = 0.0;
        for (int64_t p = 0; p < P->n_paths; ++p) {
            const ppath *pp = &P->p[p];
            const pelem *el = P->el + pp->el_begin;
            int d = pp->d;
            for (int j = 0; j < d; ++j) o[j] = satisfied(&el[j], x);
            for (int i = 0; i < d; ++i)
                for (int j = i + 1; j < d; ++j)
                    for (int k = j + 1; k < d; ++k) {
                        int n = 0;
                        for (int l = 0; l < d; ++l) {
                            if (l == i || l == j || l == k) continue;
                            zz[n] = el[l].z;
                            oo[n] = o[l];
                            ++n;
                        }
                        double I = bernstein_integral(zz, oo, n, scr);
                        double v = pp->val * (o[i] - el[i].z) * (o[j] - el[j].z) * (o[k] - el[k].z) * I;
                        int a = el[i].feat, b = el[j].feat, c = el[k].feat;
                        out[a * F2 + b * F + c] += v; out[a * F2 + c * F + b] += v;
                        out[b * F2 + a * F + c] += v; out[b * F2 + c * F + a] += v;
                        out[c * F2 + a * F + b] += v; out[c * F2 + b * F + a] += v;
                    }
        }
    }
    free(o); free(zz); free(oo); free(scr);
    return NULL;
}

int orc_sii3_exact(const orc_ens *e, const float *X, int64_t M, int n_threads, double *sii3) {
    paths_t P;
    if (build_paths(e, &P)) return -1;
    job_t proto;
    memset(&proto, 0, sizeof(proto));
    proto.e = e; proto.P = &P; proto.X = X; proto.F = e->n_features; proto.sii = sii3;
    int rc = run_threads(sii3_exact_worker, &proto, M, n_threads);
    free_paths(&P);
    return rc;
}

/* SII_ijk = sum_{T subset of [F]\{i,j,k}} |T|! (F-|T|-3)! / (F-2)! Delta_ijk f(T),
 * Delta_ijk f(T) = sum_{L subset of {i,j,k}} (-1)^(3-|L|) f(T + L)  (App. C, |S| = 3). */
int orc_brute_force3(const orc_ens *e, const float *x, double *sii3) {
    int F = e->n_features;
    if (F < 3 || F > 16) return -1;
    uint32_t NS = 1u << F;
    double *fs = (double *)malloc(sizeof(double) * NS);
    if (!fs) return -1;
    for (uint32_t S = 0; S < NS; ++S) {
        double acc = 0.0;
        for (int t = 0; t < e->n_trees; ++t) acc += game(e, e->node_offsets[t], 0, x, S);
        fs[S] = acc;
    }
    double fact[32];
    fact[0] = 1.0;
    for (int k = 1; k < 32; ++k) fact[k] = fact[k - 1] * (double)k;
    int64_t F2 = (int64_t)F * F;
    for (int64_t q = 0; q < F2 * F; ++q) sii3[q] = 0.0;
    for (int i = 0; i < F; ++i)
        for (int j = i + 1; j < F; ++j)
            for (int k = j + 1; k < F; ++k) {
                uint32_t mi = 1u << i, mj = 1u << j, mk = 1u << k, mall = mi | mj | mk;
                double acc = 0.0;
                for (uint32_t T = 0; T < NS; ++T) {
                    if (T & mall) continue;
                    int t = __builtin_popcount(T);
                    double delta = fs[T | mall] - fs[T | mi | mj] - fs[T | mi | mk] - fs[T | mj | mk] +
                                   fs[T | mi] + fs[T | mj] + fs[T | mk] - fs[T];
                    acc += fact[t] * fact[F - t - 3] / fact[F - 2] * delta;
                }
                sii3[i * F2 + j * F + k] = acc; sii3[i * F2 + k * F + j] = acc;
                sii3[j * F2 + i * F + k] = acc; sii3[j * F2 + k * F + i] = acc;
                sii3[k * F2 + i * F + j] = acc; sii3[k * F2 + j * F + i] = acc;
            }
    free(fs);
    return 0;
}
