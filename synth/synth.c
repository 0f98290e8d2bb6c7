/*
 * Seeded synthetic inputs: random-split trees, sample matrices, batch draws.
 * Input manufacturing only; no Shapley arithmetic lives here (see synth.h).
 * Build with -ffp-contract=off so every host produces the same bits.
 */
#include "synth.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- RNG --- */

static inline uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ULL;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBULL;
    x ^= x >> 31;
    return x;
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return mix64(seed ^ mix64(stream + 0x632BE59BD9B4E019ULL));
}

static inline uint64_t rng_u64(uint64_t key, uint64_t ctr) {
    return mix64(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}

/* uniform in (0,1): 53 random bits, offset by half an ulp so 0 never occurs */
static inline double u01(uint64_t key, uint64_t ctr) {
    return ((double)(rng_u64(key, ctr) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

double synth_uniform(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return u01(stream_key(seed, stream), ctr);
}

/* Natural log for x > 0 from frexp and the atanh series
 *   ln m = 2 * sum_k y^(2k+1)/(2k+1),  y = (m-1)/(m+1),  m in [sqrt(1/2), sqrt(2)).
 * Used only to shape random numbers; written out so it is identical on every host. */
static double series_log(double x) {
    int e;
    double m = frexp(x, &e); /* x = m * 2^e, m in [0.5, 1) */
    if (m < 0.70710678118654752440) {
        m *= 2.0;
        e -= 1;
    }
    double y = (m - 1.0) / (m + 1.0);
    double y2 = y * y, term = y, sum = 0.0;
    for (int k = 0; k < 40; ++k) {
        double add = term / (double)(2 * k + 1);
        sum += add;
        if (add < 1e-18 * (sum > 0 ? sum : -sum)) break;
        term *= y2;
    }
    return 2.0 * sum + (double)e * 0.69314718055994530942;
}

/* exp(x) for moderate |x| by range reduction to |r| <= ln2/2 and a Taylor sum. */
static double series_exp(double x) {
    double kf = x / 0.69314718055994530942;
    long k = (long)(kf >= 0 ? kf + 0.5 : kf - 0.5);
    double r = x - (double)k * 0.69314718055994530942;
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 30; ++i) {
        term *= r / (double)i;
        sum += term;
    }
    return ldexp(sum, (int)k);
}

/* Marsaglia polar method: one normal per call; *ctr advances by the draws used. */
static double normal_draw(uint64_t key, uint64_t *ctr) {
    for (;;) {
        double v1 = 2.0 * u01(key, (*ctr)++) - 1.0;
        double v2 = 2.0 * u01(key, (*ctr)++) - 1.0;
        double s = v1 * v1 + v2 * v2;
        if (s >= 1.0 || s == 0.0) continue;
        return v1 * sqrt(-2.0 * series_log(s) / s);
    }
}

/* ------------------------------------------------------ normal matrix --- */

typedef struct {
    uint64_t seed, stream;
    int64_t begin, end;
    float *out;
} normal_job;

#define NORMAL_BLOCK 4096

static void *normal_worker(void *arg) {
    normal_job *j = (normal_job *)arg;
    /* each block of NORMAL_BLOCK outputs has its own counter stream, so the
     * result does not depend on how blocks are spread over threads */
    for (int64_t b = j->begin; b < j->end; b += NORMAL_BLOCK) {
        uint64_t key = stream_key(j->seed, j->stream * 0x100000001B3ULL + (uint64_t)(b / NORMAL_BLOCK));
        uint64_t ctr = 0;
        int64_t e = b + NORMAL_BLOCK < j->end ? b + NORMAL_BLOCK : j->end;
        for (int64_t i = b; i < e; ++i) j->out[i] = (float)normal_draw(key, &ctr);
    }
    return NULL;
}

void synth_normal_f32(uint64_t seed, uint64_t stream, int64_t n, int n_threads, float *out) {
    if (n <= 0) return;
    if (n_threads < 1) n_threads = 1;
    int64_t nblocks = (n + NORMAL_BLOCK - 1) / NORMAL_BLOCK;
    if (n_threads > nblocks) n_threads = (int)nblocks;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    normal_job *jobs = (normal_job *)malloc(sizeof(normal_job) * n_threads);
    int64_t per = (nblocks + n_threads - 1) / n_threads;
    for (int t = 0; t < n_threads; ++t) {
        int64_t b0 = t * per * NORMAL_BLOCK, b1 = (t + 1) * per * NORMAL_BLOCK;
        if (b1 > n) b1 = n;
        jobs[t] = (normal_job){seed, stream, b0 < n ? b0 : n, b1, out};
        pthread_create(&th[t], NULL, normal_worker, &jobs[t]);
    }
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
}

/* ------------------------------------------------------- tree growing --- */

typedef struct {
    int32_t *left, *right, *feature, *cover, *rows;
    float *threshold, *leaf_value, *z;
    uint8_t *default_left;
    int64_t n, cap;
    int32_t max_depth_seen;
} tree_buf;

static int tree_push(tree_buf *t) {
    if (t->n == t->cap) {
        int64_t c = t->cap ? 2 * t->cap : 64;
#define GROW(f, T)                                              \
    do {                                                        \
        T *p = (T *)realloc(t->f, sizeof(T) * (size_t)c);       \
        if (!p) return -1;                                      \
        t->f = p;                                               \
    } while (0)
        GROW(left, int32_t); GROW(right, int32_t); GROW(feature, int32_t);
        GROW(cover, int32_t); GROW(rows, int32_t); GROW(threshold, float);
        GROW(leaf_value, float); GROW(z, float); GROW(default_left, uint8_t);
#undef GROW
        t->cap = c;
    }
    int64_t i = t->n++;
    t->left[i] = t->right[i] = t->feature[i] = -1;
    t->cover[i] = 0;
    t->rows[i] = 0;
    t->threshold[i] = 0.f;
    t->leaf_value[i] = 0.f;
    t->z[i] = 1.f;
    t->default_left[i] = 0;
    return (int)i;
}

static void tree_release(tree_buf *t) {
    free(t->left); free(t->right); free(t->feature); free(t->cover); free(t->rows);
    free(t->threshold); free(t->leaf_value); free(t->z); free(t->default_left);
    memset(t, 0, sizeof(*t));
}

/* k-th smallest (0-based) of v[0..n) by quickselect with a median-of-three pivot;
 * reorders v.  Any correct selection gives the same value. */
static float select_kth(float *v, int64_t n, int64_t k) {
    int64_t lo = 0, hi = n - 1;
    while (hi > lo) {
        int64_t mid = lo + (hi - lo) / 2;
        float a = v[lo], b = v[mid], c = v[hi];
        float piv = (a < b) ? ((b < c) ? b : (a < c ? c : a)) : ((a < c) ? a : (b < c ? c : b));
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (v[i] < piv) ++i;
            while (v[j] > piv) --j;
            if (i <= j) {
                float t = v[i]; v[i] = v[j]; v[j] = t;
                ++i; --j;
            }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else return v[k];
    }
    return v[k];
}

typedef struct {
    int node, depth;
    int64_t lo, hi; /* range in the row-index array */
} grow_task;

typedef struct {
    uint64_t seed;
    int max_depth, min_rows, full_depth, n_features, n_train;
    double leaf_std;
    const float *train; /* column-major [n_features][n_train] */
} grow_cfg;

static int grow_tree(const grow_cfg *c, int tree_idx, tree_buf *t, int32_t *rowidx,
                     float *scratch, grow_task *stack) {
    uint64_t key = stream_key(c->seed, 0x7472656500000000ULL + (uint64_t)tree_idx);
    uint64_t ctr = 0;
    for (int i = 0; i < c->n_train; ++i) rowidx[i] = i;
    int root = tree_push(t);
    if (root < 0) return -2;
    int sp = 0;
    stack[sp++] = (grow_task){root, 0, 0, c->n_train};
    while (sp > 0) {
        grow_task g = stack[--sp];
        int64_t n = g.hi - g.lo;
        if (g.depth > t->max_depth_seen) t->max_depth_seen = g.depth;
        t->rows[g.node] = (int32_t)n;
        int leaf = g.depth >= c->max_depth || (!c->full_depth && n <= c->min_rows);
        if (leaf) {
            t->leaf_value[g.node] = (float)(c->leaf_std * normal_draw(key, &ctr));
            continue;
        }
        int f = (int)(u01(key, ctr++) * c->n_features);
        if (f >= c->n_features) f = c->n_features - 1;
        double uq = u01(key, ctr++);
        const float *col = c->train + (int64_t)f * c->n_train;
        float thr;
        if (n > 0) {
            for (int64_t i = 0; i < n; ++i) scratch[i] = col[rowidx[g.lo + i]];
            int64_t k = (int64_t)(uq * (double)n);
            if (k >= n) k = n - 1;
            thr = select_kth(scratch, n, k);
        } else {
            for (int64_t i = 0; i < c->n_train; ++i) scratch[i] = col[i];
            int64_t k = (int64_t)(uq * (double)c->n_train);
            if (k >= c->n_train) k = c->n_train - 1;
            thr = select_kth(scratch, c->n_train, k);
        }
        /* stable-enough in-place partition: x < thr to the front */
        int64_t mid = g.lo;
        for (int64_t i = g.lo; i < g.hi; ++i) {
            if (col[rowidx[i]] < thr) {
                int32_t tmp = rowidx[i]; rowidx[i] = rowidx[mid]; rowidx[mid] = tmp;
                ++mid;
            }
        }
        t->feature[g.node] = f;
        t->threshold[g.node] = thr;
        t->default_left[g.node] = (uint8_t)(u01(key, ctr++) < 0.5);
        int l = tree_push(t);
        if (l < 0) return -2;
        int r = tree_push(t);
        if (r < 0) return -2;
        t->left[g.node] = l;
        t->right[g.node] = r;
        stack[sp++] = (grow_task){r, g.depth + 1, mid, g.hi};
        stack[sp++] = (grow_task){l, g.depth + 1, g.lo, mid};
    }
    /* covers bottom-up: children always have larger indices than their parent */
    for (int64_t i = t->n - 1; i >= 0; --i) {
        if (t->left[i] < 0) t->cover[i] = t->rows[i] > 0 ? t->rows[i] : 1;
        else t->cover[i] = t->cover[t->left[i]] + t->cover[t->right[i]];
    }
    for (int64_t i = 0; i < t->n; ++i) {
        if (t->left[i] >= 0) {
            t->z[t->left[i]] = (float)((double)t->cover[t->left[i]] / (double)t->cover[i]);
            t->z[t->right[i]] = (float)((double)t->cover[t->right[i]] / (double)t->cover[i]);
        }
    }
    t->z[0] = 1.f;
    return 0;
}

typedef struct {
    const grow_cfg *cfg;
    int tid, nth, n_trees;
    tree_buf *trees;
    int status;
} grow_job;

static void *grow_worker(void *arg) {
    grow_job *j = (grow_job *)arg;
    const grow_cfg *c = j->cfg;
    int64_t nt = c->n_train > 0 ? c->n_train : 1;
    int32_t *rowidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)nt);
    float *scratch = (float *)malloc(sizeof(float) * (size_t)nt);
    /* depth-first stack never holds more than 2 entries per level */
    grow_task *stack = (grow_task *)malloc(sizeof(grow_task) * (size_t)(2 * c->max_depth + 4));
    j->status = (rowidx && scratch && stack) ? 0 : -2;
    for (int t = j->tid; t < j->n_trees && j->status == 0; t += j->nth)
        j->status = grow_tree(c, t, &j->trees[t], rowidx, scratch, stack);
    free(rowidx);
    free(scratch);
    free(stack);
    return NULL;
}

int synth_grow(uint64_t seed, int n_trees, int max_depth, int min_rows, int full_depth,
               int n_features, int n_train, double leaf_std, int n_threads, synth_ens *out) {
    if (!out || n_trees <= 0 || max_depth < 0 || max_depth > 62 || n_features <= 0 || n_train <= 0)
        return -1;
    memset(out, 0, sizeof(*out));
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_trees) n_threads = n_trees;

    float *train = (float *)malloc(sizeof(float) * (size_t)n_train * (size_t)n_features);
    if (!train) return -2;
    /* training rows: one stream per feature column */
    for (int f = 0; f < n_features; ++f)
        synth_normal_f32(seed, 0x747261696E000000ULL + (uint64_t)f, n_train, n_threads,
                         train + (int64_t)f * n_train);

    grow_cfg cfg = {seed, max_depth, min_rows, full_depth, n_features, n_train, leaf_std, train};
    tree_buf *trees = (tree_buf *)calloc((size_t)n_trees, sizeof(tree_buf));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    grow_job *jobs = (grow_job *)malloc(sizeof(grow_job) * n_threads);
    if (!trees || !th || !jobs) {
        free(train); free(trees); free(th); free(jobs);
        return -2;
    }
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = (grow_job){&cfg, t, n_threads, n_trees, trees, 0};
        pthread_create(&th[t], NULL, grow_worker, &jobs[t]);
    }
    int status = 0;
    for (int t = 0; t < n_threads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].status) status = jobs[t].status;
    }
    free(th);
    free(jobs);
    free(train);

    if (status == 0) {
        int64_t total = 0;
        for (int t = 0; t < n_trees; ++t) total += trees[t].n;
        out->n_trees = n_trees;
        out->n_features = n_features;
        out->n_nodes = total;
        out->node_offsets = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_trees + 1));
        out->left = (int32_t *)malloc(sizeof(int32_t) * (size_t)total);
        out->right = (int32_t *)malloc(sizeof(int32_t) * (size_t)total);
        out->feature = (int32_t *)malloc(sizeof(int32_t) * (size_t)total);
        out->cover = (int32_t *)malloc(sizeof(int32_t) * (size_t)total);
        out->threshold = (float *)malloc(sizeof(float) * (size_t)total);
        out->z = (float *)malloc(sizeof(float) * (size_t)total);
        out->leaf_value = (float *)malloc(sizeof(float) * (size_t)total);
        out->default_left = (uint8_t *)malloc((size_t)total);
        if (!out->node_offsets || !out->left || !out->right || !out->feature || !out->cover ||
            !out->threshold || !out->z || !out->leaf_value || !out->default_left) {
            status = -2;
        } else {
            int64_t off = 0;
            for (int t = 0; t < n_trees; ++t) {
                tree_buf *b = &trees[t];
                out->node_offsets[t] = off;
                memcpy(out->left + off, b->left, sizeof(int32_t) * b->n);
                memcpy(out->right + off, b->right, sizeof(int32_t) * b->n);
                memcpy(out->feature + off, b->feature, sizeof(int32_t) * b->n);
                memcpy(out->cover + off, b->cover, sizeof(int32_t) * b->n);
                memcpy(out->threshold + off, b->threshold, sizeof(float) * b->n);
                memcpy(out->z + off, b->z, sizeof(float) * b->n);
                memcpy(out->leaf_value + off, b->leaf_value, sizeof(float) * b->n);
                memcpy(out->default_left + off, b->default_left, b->n);
                if (b->max_depth_seen > out->max_depth_seen) out->max_depth_seen = b->max_depth_seen;
                off += b->n;
            }
            out->node_offsets[n_trees] = off;
        }
    }
    for (int t = 0; t < n_trees; ++t) tree_release(&trees[t]);
    free(trees);
    if (status) synth_free(out);
    return status;
}

void synth_free(synth_ens *e) {
    if (!e) return;
    free(e->node_offsets); free(e->left); free(e->right); free(e->feature); free(e->cover);
    free(e->threshold); free(e->z); free(e->leaf_value); free(e->default_left);
    memset(e, 0, sizeof(*e));
}

/* ------------------------------------------------------- batch draws --- */

static int loguniform_int(uint64_t key, uint64_t ctr, int lo, int hi) {
    double u = u01(key, ctr);
    double v = series_exp(series_log((double)lo) + u * (series_log((double)hi) - series_log((double)lo)));
    int r = (int)(v + 0.5);
    if (r < lo) r = lo;
    if (r > hi) r = hi;
    return r;
}

void synth_batch_draw(uint64_t seed, int n_ens, int trees_lo, int trees_hi, int depth_lo,
                      int depth_hi, int f_lo, int f_hi, int m_lo, int m_hi, int32_t *trees,
                      int32_t *depth, int32_t *nfeat, int32_t *nsamp) {
    uint64_t key = stream_key(seed, 0x6261746368000000ULL);
    for (int e = 0; e < n_ens; ++e) {
        uint64_t c = (uint64_t)e * 8;
        trees[e] = loguniform_int(key, c + 0, trees_lo, trees_hi);
        int d = depth_lo + (int)(u01(key, c + 1) * (double)(depth_hi - depth_lo + 1));
        depth[e] = d > depth_hi ? depth_hi : d;
        nfeat[e] = loguniform_int(key, c + 2, f_lo, f_hi);
        nsamp[e] = loguniform_int(key, c + 3, m_lo, m_hi);
    }
}
