// Host-side preparation: path extraction and per-feature merging (Sec. 2,
// Eq. R_empty and Eq. q_def), length bucketing into SoA tables, and the
// Gauss-Legendre rule (Sec. 4).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

#include "qts_internal.h"

namespace qts {

int bucket_width_for(int d) {
    if (d <= 16) return d;
    if (d <= 32) return (d + 3) / 4 * 4;
    return (d + 7) / 8 * 8;
}

// ------------------------------------------------------------ GL nodes ----
//
// Golub-Welsch: the n-point Gauss-Legendre nodes on [-1,1] are the eigenvalues
// of the symmetric tridiagonal Jacobi matrix with zero diagonal and
// off-diagonal k / sqrt(4k^2 - 1), k = 1..n-1; the weights are 2 v_0^2 with v
// the normalised eigenvector.  The eigenproblem is solved with cyclic Jacobi
// rotations on the dense matrix (n <= 64), then mapped to [0,1].
bool gauss_legendre(int n, double* t, double* w) {
    if (n < 1 || n > 64) return false;
    std::vector<double> A((size_t)n * n, 0.0), V((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int k = 1; k < n; ++k) {
        double b = k / std::sqrt(4.0 * k * k - 1.0);
        A[(size_t)(k - 1) * n + k] = b;
        A[(size_t)k * n + (k - 1)] = b;
    }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off < 1e-34) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                // rotation angle that annihilates A[p][q]
                double theta = (aqq - app) / (2.0 * apq);
                double tt = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(tt * tt + 1.0), s = tt * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {  // accumulate eigenvectors
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    std::vector<std::pair<double, double>> nw(n);
    for (int i = 0; i < n; ++i) {
        double v0 = V[(size_t)0 * n + i];
        nw[i] = {A[(size_t)i * n + i], 2.0 * v0 * v0};
    }
    std::sort(nw.begin(), nw.end());
    for (int i = 0; i < n; ++i) {
        t[i] = 0.5 * (nw[i].first + 1.0);
        w[i] = 0.5 * nw[i].second;
    }
    // symmetrise (the rule is symmetric about 1/2) to remove rotation noise
    for (int i = 0; i < n / 2; ++i) {
        double tl = 0.5 * (t[i] + (1.0 - t[n - 1 - i]));
        double wl = 0.5 * (w[i] + w[n - 1 - i]);
        t[i] = tl;
        t[n - 1 - i] = 1.0 - tl;
        w[i] = w[n - 1 - i] = wl;
    }
    if (n % 2 == 1) t[n / 2] = 0.5;
    return true;
}

bool make_quad(int n, QuadF* qf, QuadD* qd, int pad) {
    // the rules for 1..QTS_MAX_QUAD points, computed once (calls choose one
    // per bucket, so this runs on every launch)
    struct Rules {
        double t[QTS_MAX_QUAD + 1][QTS_MAX_QUAD], w[QTS_MAX_QUAD + 1][QTS_MAX_QUAD];
        bool ok[QTS_MAX_QUAD + 1];
    };
    static const Rules* rules = [] {
        Rules* r = new Rules();
        for (int k = 1; k <= QTS_MAX_QUAD; ++k) r->ok[k] = gauss_legendre(k, r->t[k], r->w[k]);
        return r;
    }();
    if (n < 1 || n > QTS_MAX_QUAD || pad < 1 || pad > 8 || !rules->ok[n]) return false;
    const double* t = rules->t[n];
    const double* w = rules->w[n];
    int npad = (n + pad - 1) / pad * pad;
    for (int i = 0; i < QTS_MAX_QUAD + 8; ++i) {
        double ti = i < n ? t[i] : 0.5, wi = i < n ? w[i] : 0.0;
        if (qf) { qf->t[i] = (float)ti; qf->w[i] = (float)wi; }
        if (qd) { qd->t[i] = ti; qd->w[i] = wi; }
    }
    if (qf) { qf->n = n; qf->n_pad = npad; }
    if (qd) { qd->n = n; qd->n_pad = npad; }
    return true;
}

// ------------------------------------------------------- path extraction --

namespace {

struct EdgeRec {
    int32_t feat;
    uint8_t went_left, def_left, is_cat;
    float thr;
    uint64_t cats;  // categorical edge: the categories that take it
    double w;
    int64_t child;  // global node index
};

struct ElemTmp {
    int32_t feat;
    uint8_t nan_ok;
    uint8_t is_cat, other_ok;  // categorical: the set is `cats`, plus "other" values if other_ok
    double z;
    float lo, hi;
    uint64_t cats;
    int32_t edge_off, edge_cnt;  // into the thread's edge list
};

// A path of the tables.  A sibling pair (pair tables only) is one path whose
// last element stands for both leaves A (left) and B (right) of node v: val =
// 1, the element's z = alpha = val_A z_A + val_B z_B, and a sample's
// d = val_A o_A + val_B o_B - alpha, where z_k and o_k are leaf k's merged
// weight and indicator for v's feature (both leaves share every other element).
struct PathTmp {
    int64_t leaf;
    double val;
    int32_t d;
    int64_t el_off;  // into the thread's element list
    int64_t leaf2 = -1;  // B (pairs)
    double val_a = 0, val_b = 0, z_a = 0, z_b = 0, alpha = 0;
    float theta = 0.f;
    uint8_t def_left = 0;
};

struct ThreadOut {
    std::vector<PathTmp> paths;
    std::vector<ElemTmp> elems;
    std::vector<int64_t> edge_node;
    std::vector<double> edge_w;
    std::vector<double> edge_cf;  // coefficient fixed at extraction (pair elements), else NaN
    std::vector<int64_t> empty_leaf;
    std::vector<double> empty_val;
    int64_t n_leaves = 0;
    int max_unique = 0;
    std::string err;
    qts_status st = QTS_OK;
};

void extract_trees(int t0, int t1, const int64_t* off, const int32_t* left, const int32_t* right,
                   const int32_t* feature, const float* thr, const uint8_t* defl, const float* z,
                   const float* leaf, const uint8_t* is_cat, const uint64_t* cat_left, bool pairs,
                   ThreadOut* out) {
    std::vector<EdgeRec> path;
    struct Item { int32_t v; int32_t depth; EdgeRec in; };
    std::vector<Item> stack;
    ElemTmp merged[kMaxD];
    std::vector<int64_t> medges[kMaxD];
    std::vector<double> mw[kMaxD];
    for (int t = t0; t < t1 && out->st == QTS_OK; ++t) {
        int64_t base = off[t];
        int64_t nt = off[t + 1] - base;
        if (left[base] < 0) {  // single-leaf tree: no split, only the bias
            if (nt != 1) {
                out->st = QTS_ERR_ARG;
                out->err = "tree " + std::to_string(t) + " has nodes that its root does not reach";
                return;
            }
            out->empty_leaf.push_back(base);
            out->empty_val.push_back((double)leaf[base]);
            out->n_leaves++;
            continue;
        }
        stack.clear();
        stack.push_back({0, 0, {}});
        int64_t visited = 0;
        while (!stack.empty()) {
            Item it = stack.back();
            stack.pop_back();
            if (++visited > nt) {
                out->st = QTS_ERR_ARG;
                out->err = "tree " + std::to_string(t) + " is not a tree (a node is reached twice)";
                return;
            }
            if (it.depth > 0) {
                if ((int64_t)path.size() < it.depth) path.resize(it.depth);
                path[it.depth - 1] = it.in;
            }
            int64_t g = base + it.v;
            // merge the splits on each feature of the first `depth` edges (Eq. q_def);
            // returns the number of elements, or -1 (error set) above kMaxD
            auto merge = [&](int depth) -> int {
                int d = 0;
                for (int k = 0; k < depth; ++k) {
                    const EdgeRec& e = path[k];
                    int slot = -1;
                    for (int j = 0; j < d; ++j)
                        if (merged[j].feat == e.feat) { slot = j; break; }
                    if (slot < 0) {
                        if (d == kMaxD) {
                            out->st = QTS_ERR_UNSUPPORTED;
                            out->err = "a path of tree " + std::to_string(t) + " has more than " +
                                       std::to_string(kMaxD) + " unique features";
                            return -1;
                        }
                        slot = d++;
                        merged[slot] = {e.feat, 1, 0, 1, 1.0, -INFINITY, INFINITY, ~0ull, 0, 0};
                        medges[slot].clear();
                        mw[slot].clear();
                    }
                    ElemTmp& m = merged[slot];
                    m.z *= e.w;
                    if (e.is_cat) {
                        // the categories that satisfy every split so far; values
                        // that are not categories only ever take right edges
                        m.is_cat = 1;
                        m.cats &= e.cats;
                        if (e.went_left) m.other_ok = 0;
                    } else if (e.went_left) {
                        m.hi = std::min(m.hi, e.thr);
                    } else {
                        m.lo = std::max(m.lo, e.thr);
                    }
                    if (e.went_left != e.def_left) m.nan_ok = 0;
                    medges[slot].push_back(e.child);
                    mw[slot].push_back(e.w);
                }
                return d;
            };
            // emit elements merged[order[0..n)] (sorted by feature) to the thread's lists
            auto emit_sorted = [&](int n, const int* idx) {
                int order[kMaxD];
                for (int j = 0; j < n; ++j) order[j] = idx[j];
                for (int j = 1; j < n; ++j) {
                    int key = order[j], k = j - 1;
                    while (k >= 0 && merged[order[k]].feat > merged[key].feat) {
                        order[k + 1] = order[k];
                        --k;
                    }
                    order[k + 1] = key;
                }
                for (int jj = 0; jj < n; ++jj) {
                    int j = order[jj];
                    ElemTmp m = merged[j];
                    m.edge_off = (int32_t)out->edge_node.size();
                    m.edge_cnt = (int32_t)medges[j].size();
                    for (size_t a = 0; a < medges[j].size(); ++a) {
                        out->edge_node.push_back(medges[j][a]);
                        out->edge_w.push_back(mw[j][a]);
                        out->edge_cf.push_back(NAN);
                    }
                    out->elems.push_back(m);
                }
            };
            if (left[g] < 0) {
                out->n_leaves++;
                const int d = merge(it.depth);
                if (d < 0) return;
                int idx[kMaxD];
                for (int j = 0; j < d; ++j) idx[j] = j;
                PathTmp p{g, (double)leaf[g], d, (int64_t)out->elems.size()};
                emit_sorted(d, idx);
                out->paths.push_back(p);
                out->max_unique = std::max(out->max_unique, d);
                continue;
            }
            const int64_t ga = base + left[g], gb = base + right[g];
            if (pairs && left[ga] < 0 && left[gb] < 0 && !(is_cat && is_cat[g])) {
                // both children are leaves of a numerical split: one pair path
                visited += 2;
                if (visited > nt) {
                    out->st = QTS_ERR_ARG;
                    out->err = "tree " + std::to_string(t) + " is not a tree (a node is reached twice)";
                    return;
                }
                out->n_leaves += 2;
                int d = merge(it.depth);
                if (d < 0) return;
                const int32_t f = feature[g];
                int prev = -1;
                for (int j = 0; j < d; ++j)
                    if (merged[j].feat == f) prev = j;
                if (prev < 0 && d == kMaxD) {
                    out->st = QTS_ERR_UNSUPPORTED;
                    out->err = "a path of tree " + std::to_string(t) + " has more than " + std::to_string(kMaxD) +
                               " unique features";
                    return;
                }
                // the pair element: v's feature merged over the path, then each child
                ElemTmp m = prev >= 0 ? merged[prev]
                                      : ElemTmp{f, 1, 0, 1, 1.0, -INFINITY, INFINITY, ~0ull, 0, 0};
                const double zp = m.z;
                const double wa = (double)z[ga], wb = (double)z[gb];
                PathTmp p{ga, 1.0, 0, 0};
                p.leaf2 = gb;
                p.val_a = (double)leaf[ga];
                p.val_b = (double)leaf[gb];
                p.z_a = zp * wa;
                p.z_b = zp * wb;
                p.alpha = p.val_a * p.z_a + p.val_b * p.z_b;
                p.theta = thr[g];
                p.def_left = defl ? (defl[g] != 0) : 1;
                int idx[kMaxD], n = 0;
                for (int j = 0; j < d; ++j)
                    if (j != prev) idx[n++] = j;
                p.el_off = (int64_t)out->elems.size();
                p.d = n + 1;
                emit_sorted(n, idx);
                // its edges: dL/dw_e = sum over the two leaves k of dL/dz_k dz_k/dw_e,
                // and dL/dz_k = val_k * (the element's z-gradient at val = 1)
                m.z = p.alpha;
                m.edge_off = (int32_t)out->edge_node.size();
                m.edge_cnt = 0;
                const std::vector<int64_t> no_edges;
                const std::vector<int64_t>& pe = prev >= 0 ? medges[prev] : no_edges;
                const std::vector<double> no_w;
                const std::vector<double>& pw = prev >= 0 ? mw[prev] : no_w;
                for (int k = 0; k < 2; ++k) {
                    const double vk = k == 0 ? p.val_a : p.val_b, wk = k == 0 ? wa : wb;
                    for (size_t a = 0; a < pe.size(); ++a) {
                        double others = wk;
                        for (size_t c = 0; c < pe.size(); ++c)
                            if (c != a) others *= pw[c];
                        out->edge_node.push_back(pe[a]);
                        out->edge_w.push_back(pw[a]);
                        out->edge_cf.push_back(vk * others);
                        ++m.edge_cnt;
                    }
                    out->edge_node.push_back(k == 0 ? ga : gb);
                    out->edge_w.push_back(wk);
                    out->edge_cf.push_back(vk * zp);
                    ++m.edge_cnt;
                }
                out->elems.push_back(m);
                out->paths.push_back(p);
                out->max_unique = std::max(out->max_unique, p.d);
                continue;
            }
            int32_t f = feature[g];
            // push right first so the left subtree is walked first
            for (int side = 1; side >= 0; --side) {
                int32_t c = side == 0 ? left[g] : right[g];
                EdgeRec e;
                e.feat = f;
                e.went_left = side == 0;
                e.def_left = defl ? (defl[g] != 0) : 1;
                e.is_cat = (is_cat && is_cat[g]) ? 1 : 0;
                e.cats = e.is_cat ? (side == 0 ? cat_left[g] : ~cat_left[g]) : ~0ull;
                e.thr = thr[g];
                e.w = (double)z[base + c];
                e.child = base + c;
                stack.push_back({c, it.depth + 1, e});
            }
        }
        if (visited != nt) {
            out->st = QTS_ERR_ARG;
            out->err = "tree " + std::to_string(t) + " has nodes that its root does not reach";
            return;
        }
    }
}

// Record fields of a merged element: numerical [lo, hi), or for a categorical
// one the category set's low and high 32 bits in lo and hi (bit patterns).
uint32_t elem_bits(const ElemTmp& m, float* lo, float* hi) {
    uint32_t bits = (uint32_t)m.feat | (m.nan_ok ? kNanOk : 0u);
    if (m.is_cat) {
        const uint32_t l = (uint32_t)(m.cats & 0xFFFFFFFFull), h = (uint32_t)(m.cats >> 32);
        std::memcpy(lo, &l, 4);
        std::memcpy(hi, &h, 4);
        return bits | kCat | (m.other_ok ? kOtherOk : 0u);
    }
    *lo = m.lo;
    *hi = m.hi;
    return bits;
}

}  // namespace

static qts_status validate(int32_t n_trees, const int64_t* off, const int32_t* left,
                           const int32_t* right, const int32_t* feature, const float* thr,
                           const float* z, const float* leaf, const uint8_t* is_cat,
                           const uint64_t* cat_left, int32_t F, std::string* err) {
    if (is_cat && !cat_left) { *err = "category_left_mask is NULL"; return QTS_ERR_ARG; }
    if (is_cat) {
        // a feature is either numerical or categorical throughout the ensemble
        std::vector<uint8_t> kind((size_t)F, 0);  // bit 0 numerical, bit 1 categorical
        for (int64_t g = 0; g < off[n_trees]; ++g) {
            if (left[g] < 0 || feature[g] < 0 || feature[g] >= F) continue;
            kind[feature[g]] |= is_cat[g] ? 2 : 1;
            if (kind[feature[g]] == 3) {
                *err = "feature " + std::to_string(feature[g]) + " has numerical and categorical splits";
                return QTS_ERR_ARG;
            }
        }
    }
    if (off[0] != 0) { *err = "tree_node_offsets[0] must be 0"; return QTS_ERR_ARG; }
    for (int t = 0; t < n_trees; ++t) {
        int64_t a = off[t], b = off[t + 1];
        if (b <= a) { *err = "tree " + std::to_string(t) + " has no nodes"; return QTS_ERR_ARG; }
        int64_t n = b - a;
        if (n > INT32_MAX) { *err = "tree too large"; return QTS_ERR_ARG; }
        // a proper binary tree: every node but the root has exactly one parent,
        // and every node is reached from the root (checked by the walk below)
        std::vector<uint8_t> parents((size_t)n, 0);
        for (int64_t g = a; g < b; ++g) {
            int32_t l = left[g], r = right[g];
            if ((l < 0) != (r < 0) || l >= n || r >= n || (l >= 0 && (l == 0 || r == 0 || l == r))) {
                *err = "bad children at node " + std::to_string(g);
                return QTS_ERR_ARG;
            }
            if (l >= 0 && (++parents[l] > 1 || ++parents[r] > 1)) {
                *err = "tree " + std::to_string(t) + " is not a tree (a node has two parents)";
                return QTS_ERR_ARG;
            }
            if (l >= 0) {
                if (feature[g] < 0 || feature[g] >= F) {
                    *err = "feature out of range at node " + std::to_string(g);
                    return QTS_ERR_ARG;
                }
                if (std::isnan(thr[g])) { *err = "NaN threshold at node " + std::to_string(g); return QTS_ERR_ARG; }
                for (int32_t c : {l, r}) {
                    float zc = z[a + c];
                    if (!(zc > 0.f && std::isfinite(zc))) {
                        *err = "edge weight z must be positive and finite at node " + std::to_string(a + c);
                        return QTS_ERR_ARG;
                    }
                }
            } else if (!std::isfinite(leaf[g])) {
                *err = "non-finite leaf value at node " + std::to_string(g);
                return QTS_ERR_ARG;
            }
        }
    }
    return QTS_OK;
}

qts_status prepare(int32_t n_trees, const int64_t* off, const int32_t* left, const int32_t* right,
                   const int32_t* feature, const float* thr, const uint8_t* defl, const float* z,
                   const float* leaf, const uint8_t* is_cat, const uint64_t* cat_left, int32_t F,
                   bool fp64, Prepared* P, std::string* err, bool pairs) {
    if (pairs && fp64) { *err = "sibling pairs are built for the FP32 tables only"; return QTS_ERR_ARG; }
    qts_status st = validate(n_trees, off, left, right, feature, thr, z, leaf, is_cat, cat_left, F, err);
    if (st != QTS_OK) return st;
    *P = Prepared();
    int64_t total_nodes = off[n_trees];
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    int nth = (int)std::min<int64_t>({(int64_t)hw, (int64_t)n_trees, std::max<int64_t>(1, total_nodes / 20000)});
    nth = std::max(1, nth);
    std::vector<ThreadOut> outs(nth);
    {
        // contiguous tree ranges with about equal node counts
        std::vector<int> cut(nth + 1, n_trees);
        cut[0] = 0;
        int ti = 0;
        for (int k = 1; k < nth; ++k) {
            int64_t target = total_nodes * k / nth;
            while (ti < n_trees && off[ti] < target) ++ti;
            cut[k] = std::max(cut[k - 1], ti);
        }
        std::vector<std::thread> th;
        for (int k = 0; k < nth; ++k)
            th.emplace_back(extract_trees, cut[k], cut[k + 1], off, left, right, feature, thr, defl,
                            z, leaf, is_cat, cat_left, pairs, &outs[k]);
        for (auto& x : th) x.join();
    }
    for (auto& o : outs)
        if (o.st != QTS_OK) { *err = o.err; return o.st; }

    // bucket sizes
    int64_t per_width[kMaxD + 1] = {0};
    for (auto& o : outs) {
        for (auto& p : o.paths) per_width[bucket_width_for(p.d)]++;
        P->n_leaves += o.n_leaves;
        P->max_unique = std::max(P->max_unique, o.max_unique);
        for (size_t i = 0; i < o.empty_leaf.size(); ++i) {
            P->empty_leaf.push_back(o.empty_leaf[i]);
            P->empty_val.push_back(o.empty_val[i]);
        }
    }
    int64_t rec_total = 0, path_total = 0, slot_total = 0;
    int bidx_of_width[kMaxD + 1];
    for (int D = 1; D <= kMaxD; ++D) {
        bidx_of_width[D] = -1;
        if (!per_width[D]) continue;
        Bucket b;
        b.D = D;
        b.n_paths = per_width[D];
        b.rec_off = rec_total;
        b.path_base = path_total;
        b.slot_base = slot_total;
        rec_total += b.n_paths * (D + 1);
        path_total += b.n_paths;
        slot_total += b.n_paths * D;
        bidx_of_width[D] = (int)P->buckets.size();
        P->buckets.push_back(b);
    }
    if ((int)P->buckets.size() > kMaxBuckets) { *err = "too many buckets"; return QTS_ERR_UNSUPPORTED; }
    P->n_paths = path_total;
    P->n_slots = slot_total;
    if (fp64) P->rec64.resize((size_t)rec_total);
    else P->rec32.resize((size_t)rec_total);
    P->path_leaf.resize((size_t)path_total);
    P->path_zprod.resize((size_t)path_total);
    P->path_val.resize((size_t)path_total);
    P->slot_edge_begin.assign((size_t)slot_total + 1, 0);
    P->slot_zexcl.assign((size_t)slot_total, 0.0);
    P->pairs = pairs;
    if (pairs) {
        P->pair_leaf2.assign((size_t)path_total, -1);
        P->pair_zprod2.assign((size_t)path_total, 0.0);
        P->pair_z.assign(2 * (size_t)path_total, 0.0);
        P->pair_gslot.assign((size_t)path_total, -1);
    }

    // fill, bucket by bucket in tree order; first count edges per slot
    std::vector<int64_t> cursor(P->buckets.size());
    for (size_t b = 0; b < P->buckets.size(); ++b) cursor[b] = 0;
    const uint32_t pad_bits = (uint32_t)F | kNanOk;
    for (auto& o : outs) {
        for (auto& p : o.paths) {
            int D = bucket_width_for(p.d);
            Bucket& b = P->buckets[bidx_of_width[D]];
            int64_t lp = cursor[bidx_of_width[D]]++;
            int64_t gp = b.path_base + lp;
            int64_t r = b.rec_off + lp * (D + 1);
            const bool pr = p.leaf2 >= 0;
            // element j of the path sits in slot j, except a pair's element
            // (its last), which sits in the last slot after any padding
            auto slot_of = [&](int j) { return (pr && j == p.d - 1) ? D - 1 : j; };
            double zprod = 1.0;  // pairs: the shared elements only
            for (int j = 0; j < (pr ? p.d - 1 : p.d); ++j) zprod *= o.elems[p.el_off + j].z;
            P->sum_unique += p.d;
            P->path_leaf[gp] = p.leaf;
            P->path_val[gp] = p.val;
            if (pr) {
                P->bias += p.val_a * zprod * p.z_a + p.val_b * zprod * p.z_b;
                P->path_zprod[gp] = zprod * p.z_a;
                P->pair_leaf2[gp] = p.leaf2;
                P->pair_zprod2[gp] = zprod * p.z_b;
                P->pair_z[2 * gp] = p.z_a;
                P->pair_z[2 * gp + 1] = p.z_b;
                P->pair_gslot[gp] = b.slot_base + lp * D + D - 1;
                ++P->n_pair_paths;
            } else {
                P->bias += p.val * zprod;
                P->path_zprod[gp] = zprod;
            }
            if (fp64) {
                P->rec64[r] = {p.val, zprod, 0.f, 0.f, 0u, 0u};
                for (int j = 0; j < D; ++j) {
                    if (j < p.d) {
                        const ElemTmp& m = o.elems[p.el_off + j];
                        float lo, hi;
                        const uint32_t bits = elem_bits(m, &lo, &hi);
                        if (m.is_cat) P->has_cat = true;
                        P->rec64[r + 1 + j] = {m.z, 0.0, lo, hi, bits, 0u};
                    } else {
                        P->rec64[r + 1 + j] = {1.0, 0.0, -INFINITY, INFINITY, pad_bits, 0u};
                    }
                }
            } else {
                if (pr) {
                    uint32_t tb;
                    std::memcpy(&tb, &p.theta, 4);
                    P->rec32[r] = {1.f, (float)(p.val_a - p.alpha), (float)(p.val_b - p.alpha), tb};
                } else {
                    P->rec32[r] = {(float)p.val, (float)zprod, 0.f, 0u};
                }
                for (int j = 0; j < D; ++j) P->rec32[r + 1 + j] = {1.f, -INFINITY, INFINITY, pad_bits};
                for (int j = 0; j < p.d; ++j) {
                    const ElemTmp& m = o.elems[p.el_off + j];
                    float lo, hi;
                    uint32_t bits = elem_bits(m, &lo, &hi);
                    if (m.is_cat) P->has_cat = true;
                    if (pr && j == p.d - 1) bits |= kPairElem | (p.def_left ? kDefLeft : 0u);
                    P->rec32[r + 1 + slot_of(j)] = {(float)m.z, lo, hi, bits};
                }
            }
            int64_t slot0 = b.slot_base + lp * D;
            for (int j = 0; j < p.d; ++j) {
                P->slot_edge_begin[slot0 + slot_of(j) + 1] = o.elems[p.el_off + j].edge_cnt;
                double ex = 1.0;  // prod of the other elements' z (no division)
                for (int l = 0; l < p.d; ++l)
                    if (l != j) ex *= o.elems[p.el_off + l].z;
                P->slot_zexcl[slot0 + slot_of(j)] = ex;
            }
        }
    }
    for (int64_t s = 0; s < slot_total; ++s) P->slot_edge_begin[s + 1] += P->slot_edge_begin[s];
    P->edge_node.resize((size_t)P->slot_edge_begin[slot_total]);
    P->edge_coef.resize((size_t)P->slot_edge_begin[slot_total]);
    for (size_t b = 0; b < P->buckets.size(); ++b) cursor[b] = 0;
    for (auto& o : outs) {
        for (auto& p : o.paths) {
            int D = bucket_width_for(p.d);
            Bucket& b = P->buckets[bidx_of_width[D]];
            int64_t lp = cursor[bidx_of_width[D]]++;
            int64_t slot0 = b.slot_base + lp * D;
            const bool pr = p.leaf2 >= 0;
            for (int j = 0; j < p.d; ++j) {
                const ElemTmp& m = o.elems[p.el_off + j];
                int64_t e0 = P->slot_edge_begin[slot0 + ((pr && j == p.d - 1) ? D - 1 : j)];
                for (int a = 0; a < m.edge_cnt; ++a) {
                    double coef = o.edge_cf[m.edge_off + a];
                    if (std::isnan(coef)) {  // the product of the element's other edge weights
                        coef = 1.0;
                        for (int c = 0; c < m.edge_cnt; ++c)
                            if (c != a) coef *= o.edge_w[m.edge_off + c];
                    }
                    P->edge_node[e0 + a] = o.edge_node[m.edge_off + a];
                    P->edge_coef[e0 + a] = coef;
                }
            }
        }
    }
    for (double v : P->empty_val) P->bias += v;
    return QTS_OK;
}

}  // namespace qts
