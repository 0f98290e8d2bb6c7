// First-order Shapley values by the depth-first traversal of Algorithm 1
// (Sec. 5), on the GPU.
//
// The path-form kernels evaluate every root-to-leaf path separately, so their
// work grows with sum over paths of the merged path length.  Algorithm 1 walks
// each tree once per sample and shares the products of a node's ancestors
// among all leaves below it, so its work grows with the number of edges.  For
// trees whose paths share long prefixes (deep trees, many leaves) that is
// several times less arithmetic.
//
// Formulation.  For a sample, a quadrature node t and a node v of the tree let
//   C_v(t) = w_m * prod over the merged features f on the root path of v of
//            a_f(t) = z_f + (o_f - z_f) t            (Thm 1 factors, Sec. 2)
// (top-down) and, for a child u of v reached through an edge on feature f,
//   G_u(t) = sum over leaves l below u of val_l * prod of the edge factors
//            between u and l                          (bottom-up)
// where the factor of an edge is a_new / a_old: the merged factor of its feature
// after the edge divided by the one before it (a_old = 1 when the feature is
// new on the path).  This is the telescoping of Eq.
// our_telescoping_background with every leaf's weight w_prod folded into the
// factors, which keeps C in [0, 1] instead of growing like 1/prod w.  The
// edge's contribution to phi_f is, summed over the quadrature nodes,
//   new feature:      (o - z) * C_v * G_u
//   repeated feature: C_v * G_u * r * ((o - z) - a_new * (o_old - z_old) * r),
//                     r = 1 / a_old
// (H_u * delta_e of Eq. our_telescoping_background with H_u = C_v * factor *
// G_u).  Only repeated features divide.
//
// GPU mapping.  A lane is a sample; all 8 nodes of a node group live in the
// lane's registers as four f32x2 pairs, so one traversal step serves 8 nodes.
// The traversal is the same for every sample (only the 0/1 edge tests differ),
// so control flow is warp-uniform.  Each internal node is one 32-byte record in
// preorder; a node's leaf children are finished at the node itself, and the
// per-lane stack in shared memory holds C_v (and G_v where the second child is
// internal) for the levels of the current path.  A warp owns 32 samples and a
// chunk of trees, accumulates phi in a private shared-memory tile in FP32 and
// adds it to the FP64 output once per chunk.
#include <algorithm>
#include <cstring>
#include <vector>

#include "qts_device.cuh"
#include "qts_internal.h"

namespace qts {

// One internal node of a tree in preorder (32 bytes).  zc[c] is the merged z of
// the split feature through child c's edge (the product of the weights of every
// edge on this feature from the root down to and including that edge), zold the
// merged z before this node (1 when the feature is new on the path), val[c] the
// leaf value of a leaf child.  meta: feature (bits 0-15), depth of the nearest
// ancestor splitting on the same feature (16-22; kDfsNoAnc when none), child 0
// is a leaf (23), child 1 is a leaf (24), NaN goes left (25).  depth: this
// node's depth (the root is 0).
struct __align__(16) DfsRec {
    float thr;
    float zc[2];
    float zold;
    float val[2];
    uint32_t meta;
    uint32_t depth;
};
constexpr uint32_t kDfsNoAnc = 127;
constexpr int kDfsMaxLevels = 63;  // per-lane level bits live in 64-bit masks
constexpr int kDfsMaxWarps = 4;    // warps per block (each owns its own shared memory)

struct DfsArgs {
    const DfsRec* rec;
    const int64_t* tree_off;
    const float* X;       // M x F row-major
    double* phi;          // M x (F+1)
    int64_t M;
    int64_t n_items;
    int32_t n_trees;
    int32_t chunk;        // trees per work item
    int32_t n_tiles;      // sample tiles of 32
    int32_t levels;       // stack levels (internal-node depth + 1)
    int32_t F;
    int32_t groups;       // node groups of 8
    int32_t warp_floats;  // shared floats per warp
    int32_t wpb;          // warps per block
    QuadF q;
};

struct DfsMeta {
    int f, anc, depth;
    bool leaf0, leaf1, dl;
};

__device__ __forceinline__ DfsMeta dfs_meta(const DfsRec& r) {
    DfsMeta m;
    m.f = (int)(r.meta & 0xFFFFu);
    m.anc = (int)((r.meta >> 16) & 0x7Fu);
    m.leaf0 = (r.meta >> 23) & 1u;
    m.leaf1 = (r.meta >> 24) & 1u;
    m.dl = (r.meta >> 25) & 1u;
    m.depth = (int)r.depth;
    return m;
}

__device__ __forceinline__ DfsRec dfs_load(const DfsRec* p) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    DfsRec r;
    r.thr = a.x;
    r.zc[0] = a.y;
    r.zc[1] = a.z;
    r.zold = a.w;
    r.val[0] = b.x;
    r.val[1] = b.y;
    r.meta = __float_as_uint(b.z);
    r.depth = __float_as_uint(b.w);
    return r;
}

// a(t) = z + d t for the four node pairs
__device__ __forceinline__ void dfs_factor(const float2 (&T)[4], float z, float d, float2 (&a)[4]) {
#pragma unroll
    for (int p = 0; p < 4; ++p) a[p] = fma2(T[p], f2s(d), f2s(z));
}

// 1 / a_old for a repeated feature.  a_old > 0 in exact arithmetic; when the
// merged z has underflowed in FP32 the subtree's products are zero anyway, and
// r = 0 keeps them zero instead of turning 0 * inf into NaN.
__device__ __forceinline__ float dfs_recip(float a) { return a > 1e-30f ? __fdividef(1.f, a) : 0.f; }

__device__ __forceinline__ void dfs_rold(const float2 (&T)[4], float zold, float dold, float2 (&r)[4]) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float2 a = fma2(T[p], f2s(dold), f2s(zold));
        r[p] = make_float2(dfs_recip(a.x), dfs_recip(a.y));
    }
}

// sum over the 8 nodes of C * G
__device__ __forceinline__ float dfs_dot(const float2 (&C)[4], const float2 (&G)[4]) {
    float2 s = mul2(C[0], G[0]);
#pragma unroll
    for (int p = 1; p < 4; ++p) s = fma2(C[p], G[p], s);
    return s.x + s.y;
}

// Contribution of one edge (summed over the nodes) and its factor, given the
// parent's C, the child's G, the edge's merged z and o, and for a repeated
// feature r = 1/a_old and d_old = o_old - z_old.
template <bool REP>
__device__ __forceinline__ float dfs_edge(const float2 (&T)[4], const float2 (&C)[4], const float2 (&G)[4],
                                          float zc, float d, const float2 (&r)[4], float dold,
                                          float2 (&factor)[4]) {
    float2 a[4];
    dfs_factor(T, zc, d, a);
    if constexpr (!REP) {
#pragma unroll
        for (int p = 0; p < 4; ++p) factor[p] = a[p];
        return d * dfs_dot(C, G);
    } else {
        float2 s = f2s(0.f);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            factor[p] = mul2(a[p], r[p]);                       // a_new / a_old
            const float2 q = mul2(r[p], fma2(f2s(-dold), factor[p], f2s(d)));
            s = fma2(mul2(C[p], G[p]), q, s);
        }
        return s.x + s.y;
    }
}

// The edge's factor alone: a_new, or a_new / a_old for a repeated feature.
template <bool REP>
__device__ __forceinline__ void dfs_edge_factor(const float2 (&T)[4], float zc, float d, const float2 (&r)[4],
                                                float2 (&factor)[4]) {
    dfs_factor(T, zc, d, factor);
    if constexpr (REP) {
#pragma unroll
        for (int p = 0; p < 4; ++p) factor[p] = mul2(factor[p], r[p]);
    }
}

// Same with G = val (a leaf child): contribution and G_parent += factor * val.
template <bool REP>
__device__ __forceinline__ float dfs_leaf(const float2 (&T)[4], const float2 (&C)[4], float zc, float d,
                                          float val, const float2 (&r)[4], float dold, float2 (&Gp)[4]) {
    const float2 V[4] = {f2s(val), f2s(val), f2s(val), f2s(val)};
    float2 factor[4];
    const float c = dfs_edge<REP>(T, C, V, zc, d, r, dold, factor);
#pragma unroll
    for (int p = 0; p < 4; ++p) Gp[p] = fma2(factor[p], V[p], Gp[p]);
    return c;
}

__device__ __forceinline__ void dfs_store(float4* stk, int level, int part, int lane, const float2 (&v)[4]) {
    float4* p = stk + ((size_t)level * 4 + part) * 32 + lane;
    p[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    p[32] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}

__device__ __forceinline__ void dfs_fetch(const float4* stk, int level, int part, int lane, float2 (&v)[4]) {
    const float4* p = stk + ((size_t)level * 4 + part) * 32 + lane;
    const float4 a = p[0], b = p[32];
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y);
    v[3] = make_float2(b.z, b.w);
}

template <typename MaskT>
__device__ __forceinline__ bool dfs_bit(MaskT m, int k) {
    return ((m >> k) & (MaskT)1) != 0;
}

template <typename MaskT>
__device__ __forceinline__ MaskT dfs_setbit(MaskT m, int k, bool v) {
    return (m & ~((MaskT)1 << k)) | ((MaskT)v << k);
}

__device__ __forceinline__ float dfs_sum(const float2 (&C)[4]) {
    const float2 s = add2(add2(C[0], C[1]), add2(C[2], C[3]));
    return s.x + s.y;
}

// One tree for the warp's 32 samples and one node group.  MaskT holds one bit
// per level (uint32_t when the trees are at most 32 internal levels deep).
template <typename MaskT>
__device__ void dfs_tree(const DfsRec* __restrict__ rec, int nrec, const float* xs, float* tile,
                         float4* stk, int* lvl, int lane, const float2 (&T)[4], const float2 (&W)[4]) {
    float2 C[4], G[4], R[4], Rp[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        C[p] = W[p];
        G[p] = f2s(0.f);
        R[p] = Rp[p] = f2s(1.f);  // only read at repeated features, where they are set
    }
    MaskT om = 0, gm = 0;  // per level: merged o of the edge taken, and "x goes left"
    DfsRec rn = dfs_load(rec);
    for (int i = 0; i < nrec; ++i) {
        const DfsRec r = rn;
        if (i + 1 < nrec) rn = dfs_load(rec + i + 1);  // next record, in flight during this one
        const DfsMeta m = dfs_meta(r);
        const float x = xs[m.f * 33 + lane];
        const bool gl = (x != x) ? m.dl : (x < r.thr);
        const bool rep = m.anc != (int)kDfsNoAnc;
        const float ol = (!rep || dfs_bit(om, m.anc)) ? 1.f : 0.f;  // merged o above the node
        const float o0 = gl ? ol : 0.f;
        const float d0 = o0 - r.zc[0], d1 = (ol - o0) - r.zc[1];
        float dold = 0.f;
        if (rep) {
            dold = ol - r.zold;
            dfs_rold(T, r.zold, dold, R);
        }
        if (m.leaf0 || m.leaf1) {
            float c;
            if (!rep) {
                // both leaf children at once: G += val (z + d t), phi_f += val d sum(C)
                const float vd = (m.leaf0 ? r.val[0] * d0 : 0.f) + (m.leaf1 ? r.val[1] * d1 : 0.f);
                const float vz = (m.leaf0 ? r.val[0] * r.zc[0] : 0.f) + (m.leaf1 ? r.val[1] * r.zc[1] : 0.f);
                c = vd * dfs_sum(C);
#pragma unroll
                for (int p = 0; p < 4; ++p) G[p] = fma2(T[p], f2s(vd), add2(G[p], f2s(vz)));
            } else {
                c = 0.f;
                if (m.leaf0) c += dfs_leaf<true>(T, C, r.zc[0], d0, r.val[0], R, dold, G);
                if (m.leaf1) c += dfs_leaf<true>(T, C, r.zc[1], d1, r.val[1], R, dold, G);
            }
            tile[m.f * 32 + lane] += c;
        }
        const int k = m.depth;
        if (!(m.leaf0 && m.leaf1)) {
            // descend into the first internal child; the next record is its
            const int side = m.leaf0 ? 1 : 0;
            dfs_store(stk, k, 0, lane, C);
            lvl[k] = i * 2 + side;
            om = dfs_setbit(om, k, (side ? (ol - o0) : o0) != 0.f);
            gm = dfs_setbit(gm, k, gl);
            const float zc = side ? r.zc[1] : r.zc[0], d = side ? d1 : d0;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                float2 a = fma2(T[p], f2s(d), f2s(zc));
                if (rep) a = mul2(a, R[p]);
                C[p] = mul2(C[p], a);
                G[p] = f2s(0.f);
            }
            continue;
        }
        // both children are leaves: this subtree is done; return upwards until
        // an ancestor has an internal right child still to visit
        int kk = k;
        while (kk > 0) {
            const int kp = kk - 1;
            const int L = lvl[kp];
            const int side = L & 1;
            const DfsRec rp = dfs_load(rec + (L >> 1));
            const DfsMeta mp = dfs_meta(rp);
            const bool repp = mp.anc != (int)kDfsNoAnc;
            const float olp = (!repp || dfs_bit(om, mp.anc)) ? 1.f : 0.f;
            const float o0p = dfs_bit(gm, kp) ? olp : 0.f;
            const float dp0 = o0p - rp.zc[0], dp1 = (olp - o0p) - rp.zc[1];
            const float ds = side ? dp1 : dp0, zs = side ? rp.zc[1] : rp.zc[0];
            const bool sib_leaf = side ? mp.leaf0 : mp.leaf1;
            float2 Cp[4], Gp[4];
            dfs_fetch(stk, kp, 0, lane, Cp);
            if (side == 1 && !mp.leaf0) {
                dfs_fetch(stk, kp, 2, lane, Gp);  // the left subtree's share, stored before the descent
            } else {
#pragma unroll
                for (int p = 0; p < 4; ++p) Gp[p] = f2s(0.f);
            }
            float c;
            if (!repp) {
                if (sib_leaf) {  // the leaf sibling's part of G_parent, recomputed
                    const float vs = side ? rp.val[0] : rp.val[1];
                    const float vd = vs * (side ? dp0 : dp1), vz = vs * (side ? rp.zc[0] : rp.zc[1]);
#pragma unroll
                    for (int p = 0; p < 4; ++p) Gp[p] = fma2(T[p], f2s(vd), add2(Gp[p], f2s(vz)));
                }
                c = ds * dfs_dot(Cp, G);
#pragma unroll
                for (int p = 0; p < 4; ++p) Gp[p] = fma2(fma2(T[p], f2s(ds), f2s(zs)), G[p], Gp[p]);
            } else {
                const float doldp = olp - rp.zold;
                dfs_rold(T, rp.zold, doldp, Rp);
                if (sib_leaf) {
                    float2 fs[4];
                    dfs_edge_factor<true>(T, side ? rp.zc[0] : rp.zc[1], side ? dp0 : dp1, Rp, fs);
                    const float2 vs = f2s(side ? rp.val[0] : rp.val[1]);
#pragma unroll
                    for (int p = 0; p < 4; ++p) Gp[p] = fma2(fs[p], vs, Gp[p]);
                }
                float2 factor[4];
                c = dfs_edge<true>(T, Cp, G, zs, ds, Rp, doldp, factor);
#pragma unroll
                for (int p = 0; p < 4; ++p) Gp[p] = fma2(factor[p], G[p], Gp[p]);
            }
            tile[mp.f * 32 + lane] += c;
            if (side == 0 && !mp.leaf1) {
                // visit the right child next (the next record)
                dfs_store(stk, kp, 2, lane, Gp);
                lvl[kp] = L | 1;
                om = dfs_setbit(om, kp, (olp - o0p) != 0.f);
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    float2 a = fma2(T[p], f2s(dp1), f2s(rp.zc[1]));
                    if (repp) a = mul2(a, Rp[p]);
                    C[p] = mul2(Cp[p], a);
                    G[p] = f2s(0.f);
                }
                break;
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                C[p] = Cp[p];
                G[p] = Gp[p];
            }
            kk = kp;
        }
    }
}

__global__ void __launch_bounds__(kDfsMaxWarps * 32) dfs_kernel(DfsArgs a) {
    extern __shared__ __align__(16) float dfs_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t item = (int64_t)blockIdx.x * a.wpb + warp;
    if (item >= a.n_items) return;  // warp-uniform
    float* base = dfs_smem + (size_t)warp * a.warp_floats;
    float4* stk = reinterpret_cast<float4*>(base);            // levels x 4 parts x 32 lanes
    float* xs = base + (size_t)a.levels * 512;                // F x 33
    float* tile = xs + (size_t)a.F * 33;                      // F x 32
    int* lvl = reinterpret_cast<int*>(tile + (size_t)a.F * 32);  // levels
    const int F = a.F;
    const int64_t ti = item % a.n_tiles, ci = item / a.n_tiles;
    const int64_t s0 = ti * 32, s = s0 + lane;
    for (int idx = lane; idx < 32 * F; idx += 32) {
        const int j = idx / F, f = idx - j * F;
        xs[f * 33 + j] = (s0 + j < a.M) ? a.X[(s0 + j) * F + f] : 0.f;
        tile[idx] = 0.f;
    }
    __syncwarp();
    const int t0 = (int)(ci * a.chunk);
    const int t1 = min(a.n_trees, t0 + a.chunk);
    for (int g = 0; g < a.groups; ++g) {
        float2 T[4], W[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            T[p] = make_float2(a.q.t[8 * g + 2 * p], a.q.t[8 * g + 2 * p + 1]);
            W[p] = make_float2(a.q.w[8 * g + 2 * p], a.q.w[8 * g + 2 * p + 1]);
        }
        for (int t = t0; t < t1; ++t) {
            const int64_t b = a.tree_off[t], n = a.tree_off[t + 1] - b;
            if (n <= 0) continue;
            if (a.levels <= 32) dfs_tree<uint32_t>(a.rec + b, (int)n, xs, tile, stk, lvl, lane, T, W);
            else dfs_tree<uint64_t>(a.rec + b, (int)n, xs, tile, stk, lvl, lane, T, W);
        }
    }
    __syncwarp();
    if (s < a.M) {
        for (int f = 0; f < F; ++f) {
            const float v = tile[f * 32 + lane];
            if (v != 0.f) atomicAdd(&a.phi[s * (F + 1) + f], (double)v);
        }
    }
}

// ------------------------------------------------------------ host program --

namespace {

// The model's node arrays, as given to the loader.
struct DfsModel {
    const int64_t* off;
    const int32_t *left, *right, *feature;
    const float *thr, *z, *leaf;
    const uint8_t* defl;
    int32_t n_trees, n_features;
};

struct DfsBuilder {
    DfsModel e;
    int64_t base;
    std::vector<DfsRec>* out;
    std::vector<double> zcur;  // merged z of each feature on the current path
    std::vector<int> anc;      // depth of the nearest ancestor split on each feature
    int max_depth = 0;
    bool too_deep = false;

    void visit(int32_t v, int depth) {
        if (depth >= kDfsMaxLevels) {
            too_deep = true;
            return;
        }
        max_depth = std::max(max_depth, depth);
        const int64_t g = base + v;
        const int f = e.feature[g];
        const int32_t ch[2] = {e.left[g], e.right[g]};
        const bool seen = anc[f] >= 0;
        const double zold = seen ? zcur[f] : 1.0;
        DfsRec r;
        r.thr = e.thr[g];
        r.zold = (float)zold;
        bool leaf[2];
        for (int c = 0; c < 2; ++c) {
            const int64_t gc = base + ch[c];
            leaf[c] = e.left[gc] < 0;
            r.zc[c] = (float)(zold * (double)e.z[gc]);
            r.val[c] = leaf[c] ? e.leaf[gc] : 0.f;
        }
        r.meta = (uint32_t)f | ((uint32_t)(seen ? anc[f] : (int)kDfsNoAnc) << 16) |
                 ((uint32_t)leaf[0] << 23) | ((uint32_t)leaf[1] << 24) | ((uint32_t)(e.defl[g] != 0) << 25);
        r.depth = (uint32_t)depth;
        out->push_back(r);
        for (int c = 0; c < 2; ++c) {
            if (leaf[c]) continue;
            const double zs = zcur[f];
            const int as = anc[f];
            zcur[f] = zold * (double)e.z[base + ch[c]];
            anc[f] = depth;
            visit(ch[c], depth + 1);
            zcur[f] = zs;
            anc[f] = as;
            if (too_deep) return;
        }
    }
};

// The preorder record program of every tree (host); recs and off are filled,
// levels receives the deepest internal node's depth + 1.
qts_status dfs_program(const DfsModel& m, std::vector<DfsRec>* recs, std::vector<int64_t>* off, int* levels) {
    recs->clear();
    off->assign((size_t)m.n_trees + 1, 0);
    DfsBuilder b;
    b.e = m;
    b.out = recs;
    b.zcur.assign((size_t)m.n_features, 1.0);
    b.anc.assign((size_t)m.n_features, -1);
    for (int t = 0; t < m.n_trees; ++t) {
        b.base = m.off[t];
        if (m.left[b.base] >= 0) b.visit(0, 0);
        if (b.too_deep)
            return fail(QTS_ERR_UNSUPPORTED, "a tree has internal nodes deeper than " +
                                                 std::to_string(kDfsMaxLevels - 1) + " (depth-first form)");
        (*off)[t + 1] = (int64_t)recs->size();
    }
    *levels = b.max_depth + 1;
    return QTS_OK;
}

}  // namespace

qts_status build_dfs_program(qts_ensemble* e) {
    if (e->d_dfs) return QTS_OK;
    if (e->left.empty()) return fail(QTS_ERR_ARG, "ensemble has no host model");
    std::vector<DfsRec> recs;
    std::vector<int64_t> off;
    int levels = 0;
    const DfsModel m{e->off.data(), e->left.data(), e->right.data(), e->feature.data(), e->thr.data(),
                     e->z.data(), e->leaf.data(), e->defl.data(), e->n_trees, e->n_features};
    qts_status st = dfs_program(m, &recs, &off, &levels);
    if (st != QTS_OK) return st;
    DfsRec* d_rec = nullptr;
    int64_t* d_off = nullptr;
    cudaError_t ce = cudaMalloc(&d_rec, std::max<size_t>(recs.size(), 1) * sizeof(DfsRec));
    if (ce == cudaSuccess) ce = cudaMalloc(&d_off, off.size() * sizeof(int64_t));
    if (ce == cudaSuccess && !recs.empty())
        ce = cudaMemcpy(d_rec, recs.data(), recs.size() * sizeof(DfsRec), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        cudaFree(d_rec);
        cudaFree(d_off);
        return cuda_fail(ce, "depth-first program upload");
    }
    e->d_dfs = d_rec;
    e->d_dfs_off = d_off;
    e->dfs_levels = levels;
    e->dfs_records = (int64_t)recs.size();
    return QTS_OK;
}

void release_dfs(qts_ensemble* e) {
    cudaFree(e->d_dfs);
    cudaFree(e->d_dfs_off);
    e->d_dfs = nullptr;
    e->d_dfs_off = nullptr;
    e->dfs_levels = 0;
    e->dfs_records = 0;
}

}  // namespace qts

using namespace qts;

extern "C" qts_status qts_shap_values_alg1(qts_ensemble* e, const float* X, int64_t M, int32_t F,
                                           int32_t n_quad, double* phi, qts_stream_t stream) {
    qts_status st = check_call(e, X, M, F, n_quad);
    if (st != QTS_OK) return st;
    if (e->flags & QTS_FLAG_FP64)
        return fail(QTS_ERR_UNSUPPORTED, "the depth-first form runs on FP32 ensembles only");
    if (!e->is_cat.empty())
        return fail(QTS_ERR_UNSUPPORTED, "the depth-first form has no categorical splits");
    if (M == 0) return QTS_OK;
    if (!phi) return fail(QTS_ERR_ARG, "phi is NULL");
    st = build_dfs_program(e);
    if (st != QTS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    QuadF qf;
    QuadD qd;
    // QTS_NQ_EXACT: exact for the ensemble's widest path (first order, Thm 2)
    if (!make_quad(nodes_for(n_quad, e->prep.max_unique, 1), &qf, &qd)) return fail(QTS_ERR_ARG, "quadrature rule");
    cudaError_t ce = launch_phi_init(phi, M, F, e->prep.bias, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "phi init launch");
    const int levels = std::max(e->dfs_levels, 1);
    const int warp_floats = ((levels * 512 + F * 33 + F * 32 + levels) + 3) & ~3;
    const size_t warp_bytes = (size_t)warp_floats * 4;
    const size_t sm_bytes = 228 * 1024, block_max = 227 * 1024, block_reserved = 1024;
    if (warp_bytes > block_max)
        return fail(QTS_ERR_UNSUPPORTED, "depth-first form: tree depth and F need " + std::to_string(warp_bytes) +
                                             " bytes of shared memory per warp");
    // warps per block: the most resident warps per SM (shared memory bound)
    int wpb = 1, resident = 0;
    for (int w = 1; w <= kDfsMaxWarps; w *= 2) {
        if (w * warp_bytes > block_max) break;
        const int r = (int)(sm_bytes / (w * warp_bytes + block_reserved)) * w;
        if (r > resident) {
            resident = r;
            wpb = w;
        }
    }
    DfsArgs a{};
    a.rec = (const DfsRec*)e->d_dfs;
    a.tree_off = e->d_dfs_off;
    a.X = X;
    a.phi = phi;
    a.M = M;
    a.n_trees = e->n_trees;
    a.n_tiles = (int32_t)((M + 31) / 32);
    a.levels = levels;
    a.F = F;
    a.groups = qf.n_pad / 8;
    a.warp_floats = warp_floats;
    a.wpb = wpb;
    a.q = qf;
    // enough work items to fill the GPU several times over: split the trees
    // into chunks when there are few sample tiles
    const int64_t target = 4LL * num_sms() * std::max(resident, 1);
    int64_t n_chunks = std::min<int64_t>(e->n_trees, std::max<int64_t>(1, (target + a.n_tiles - 1) / a.n_tiles));
    a.chunk = (int32_t)((e->n_trees + n_chunks - 1) / n_chunks);
    n_chunks = (e->n_trees + a.chunk - 1) / a.chunk;
    a.n_items = (int64_t)a.n_tiles * n_chunks;
    const size_t smem = warp_bytes * wpb;
    if (smem > 48 * 1024) {
        ce = cudaFuncSetAttribute(dfs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ce != cudaSuccess) return cuda_fail(ce, "depth-first kernel attribute");
    }
    const int64_t blocks = (a.n_items + wpb - 1) / wpb;
    if (blocks > INT32_MAX) return fail(QTS_ERR_UNSUPPORTED, "depth-first form: too many work items");
    dfs_kernel<<<(unsigned)blocks, wpb * 32, smem, s>>>(a);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_fail(ce, "depth-first kernel launch");
    return QTS_OK;
}

extern "C" qts_status qts_describe_alg1_program(int32_t n_trees, const int64_t* off, const int32_t* left,
                                                const int32_t* right, const int32_t* feature,
                                                const float* threshold, const uint8_t* default_left,
                                                const float* z, const float* leaf_value, int32_t n_features,
                                                int64_t* n_records, uint32_t* records, int64_t* tree_off,
                                                int32_t* levels) {
    if (!n_records || n_trees < 1 || !off || !left || !right || !feature || !threshold || !z || !leaf_value)
        return fail(QTS_ERR_ARG, "NULL argument or n_trees < 1");
    if (n_features < 1 || n_features > QTS_MAX_FEATURES)
        return fail(QTS_ERR_UNSUPPORTED, "n_features out of range");
    for (int t = 0; t < n_trees; ++t)
        if (off[t + 1] <= off[t]) return fail(QTS_ERR_ARG, "tree_node_offsets must be increasing");
    // the same validation as the loader (path preparation also checks the trees)
    std::vector<uint8_t> defl;
    if (!default_left) defl.assign((size_t)off[n_trees], 1);
    const uint8_t* dl = default_left ? default_left : defl.data();
    Prepared P;
    std::string err;
    qts_status st = prepare(n_trees, off, left, right, feature, threshold, dl, z, leaf_value, nullptr, nullptr,
                            n_features, false, &P, &err);
    if (st != QTS_OK) return fail(st, err);
    std::vector<DfsRec> recs;
    std::vector<int64_t> toff;
    int lv = 0;
    const DfsModel m{off, left, right, feature, threshold, z, leaf_value, dl, n_trees, n_features};
    st = dfs_program(m, &recs, &toff, &lv);
    if (st != QTS_OK) return st;
    *n_records = (int64_t)recs.size();
    if (!records) return QTS_OK;
    if (!tree_off || !levels) return fail(QTS_ERR_ARG, "tree_off or levels is NULL");
    std::memcpy(records, recs.data(), recs.size() * sizeof(DfsRec));
    std::memcpy(tree_off, toff.data(), toff.size() * sizeof(int64_t));
    *levels = lv;
    return QTS_OK;
}
