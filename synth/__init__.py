"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

Only input manufacturing lives here: random-split regression trees grown on
synthetic N(0,1) training rows (covers = rows routed, edge weight
z = cover(child)/cover(parent) as in Sec. 2 of the paper), N(0,1) sample
matrices and the size draws of the heterogeneous batch.  No Shapley arithmetic.

The five workloads mirror the paper's XGBoost ensembles (Table 1) in shape:
  0  10 trees, full depth 4, F=8, M=100, 1,000 training rows, leaves ~N(0,1)
  1  1,000 trees, depth <= 8, F=50, M=10,000, 100,000 rows, leaves ~N(0,0.1^2)
  2  200 trees, depth <= 20, F=24, M=5,000, 200,000 rows (repeated features)
  3  500 trees, depth <= 6, F=30, M=2,000, 50,000 rows (pairwise interactions)
  4  64 ensembles: trees log-U[10,2000], depth U{3..16}, F log-U[8,200],
     M log-U[1,50000], training rows min(100000, 20*2^depth), grad_phi ~N(0,1)
Trees other than 0 stop splitting at depth or at <= 5 rows.  Seed = 20260500 + index.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libqts_synth.so")
_SRC = os.path.join(_HERE, "synth.c")
_lib = None

SEED_BASE = 20260500
STREAM_X = 0x5800000000
STREAM_GRAD = 0x4700000000


def build(force: bool = False) -> str:
    """Compile the generator with gcc (host code; identical bits on x86 and Arm)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "synth.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Ens(ctypes.Structure):
    _fields_ = [
        ("n_trees", ctypes.c_int32),
        ("n_features", ctypes.c_int32),
        ("n_nodes", ctypes.c_int64),
        ("node_offsets", ctypes.POINTER(ctypes.c_int64)),
        ("left", ctypes.POINTER(ctypes.c_int32)),
        ("right", ctypes.POINTER(ctypes.c_int32)),
        ("feature", ctypes.POINTER(ctypes.c_int32)),
        ("threshold", ctypes.POINTER(ctypes.c_float)),
        ("default_left", ctypes.POINTER(ctypes.c_uint8)),
        ("z", ctypes.POINTER(ctypes.c_float)),
        ("leaf_value", ctypes.POINTER(ctypes.c_float)),
        ("cover", ctypes.POINTER(ctypes.c_int32)),
        ("max_depth_seen", ctypes.c_int32),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.synth_grow.restype = ctypes.c_int
        lib.synth_grow.argtypes = [
            ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_Ens),
        ]
        lib.synth_free.argtypes = [ctypes.POINTER(_Ens)]
        lib.synth_normal_f32.argtypes = [
            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
        ]
        lib.synth_uniform.restype = ctypes.c_double
        lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.synth_batch_draw.argtypes = [ctypes.c_uint64] + [ctypes.c_int] * 9 + [i32p] * 4
        _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


class Ensemble:
    """Node arrays of a tree ensemble (host numpy).  Node indices are local to
    each tree; tree t owns nodes [node_offsets[t], node_offsets[t+1])."""

    def __init__(self, node_offsets, left, right, feature, threshold, default_left, z,
                 leaf_value, cover, n_features, max_depth_seen=None, is_cat=None, cat_left=None):
        self.node_offsets = np.ascontiguousarray(node_offsets, dtype=np.int64)
        self.left = np.ascontiguousarray(left, dtype=np.int32)
        self.right = np.ascontiguousarray(right, dtype=np.int32)
        self.feature = np.ascontiguousarray(feature, dtype=np.int32)
        self.threshold = np.ascontiguousarray(threshold, dtype=np.float32)
        self.default_left = np.ascontiguousarray(default_left, dtype=np.uint8)
        self.z = np.ascontiguousarray(z, dtype=np.float32)
        self.leaf_value = np.ascontiguousarray(leaf_value, dtype=np.float32)
        self.cover = np.ascontiguousarray(cover, dtype=np.int32)
        self.n_features = int(n_features)
        self.max_depth_seen = max_depth_seen
        # categorical splits (None: all splits numerical): is_cat[n] = 1 makes
        # node n's split categorical, cat_left[n] the categories 0..63 going left
        self.is_cat = None if is_cat is None else np.ascontiguousarray(is_cat, dtype=np.uint8)
        self.cat_left = None if cat_left is None else np.ascontiguousarray(cat_left, dtype=np.uint64)

    @property
    def n_trees(self) -> int:
        return len(self.node_offsets) - 1

    @property
    def n_nodes(self) -> int:
        return int(self.node_offsets[-1])

    @property
    def n_leaves(self) -> int:
        return int(np.count_nonzero(self.left < 0))

    def tree(self, t: int) -> "Ensemble":
        a, b = self.node_offsets[t], self.node_offsets[t + 1]
        cat = self.is_cat is not None
        return Ensemble([0, b - a], self.left[a:b], self.right[a:b], self.feature[a:b],
                        self.threshold[a:b], self.default_left[a:b], self.z[a:b],
                        self.leaf_value[a:b], self.cover[a:b], self.n_features,
                        is_cat=self.is_cat[a:b] if cat else None,
                        cat_left=self.cat_left[a:b] if cat else None)

    def subset(self, trees) -> "Ensemble":
        parts = [self.tree(int(t)) for t in trees]
        return concat(parts)

    def copy(self) -> "Ensemble":
        return Ensemble(self.node_offsets.copy(), self.left.copy(), self.right.copy(),
                        self.feature.copy(), self.threshold.copy(), self.default_left.copy(),
                        self.z.copy(), self.leaf_value.copy(), self.cover.copy(), self.n_features,
                        self.max_depth_seen,
                        is_cat=None if self.is_cat is None else self.is_cat.copy(),
                        cat_left=None if self.cat_left is None else self.cat_left.copy())


def concat(parts) -> Ensemble:
    """The trees of every part, in order, as one ensemble (each part may hold
    several trees)."""
    offs = [0]
    for p in parts:
        base = offs[-1]
        offs.extend(int(base + o) for o in p.node_offsets[1:])
    cat = lambda name: np.concatenate([getattr(p, name) for p in parts])
    kw = {}
    if any(p.is_cat is not None for p in parts):
        kw["is_cat"] = np.concatenate([p.is_cat if p.is_cat is not None else np.zeros(p.n_nodes, np.uint8)
                                       for p in parts])
        kw["cat_left"] = np.concatenate([p.cat_left if p.cat_left is not None
                                         else np.zeros(p.n_nodes, np.uint64) for p in parts])
    return Ensemble(np.array(offs, dtype=np.int64), cat("left"), cat("right"), cat("feature"),
                    cat("threshold"), cat("default_left"), cat("z"), cat("leaf_value"),
                    cat("cover"), max(p.n_features for p in parts), **kw)


def make_categorical(ens: Ensemble, features, n_categories: int, seed: int) -> Ensemble:
    """A copy of `ens` whose splits on `features` are categorical: each such
    node sends a random non-empty proper subset of the categories 0..n-1 left
    (numpy PCG64 stream `seed`).  Edge weights are kept as they are (any
    positive weights are valid inputs)."""
    out = ens.copy()
    rng = np.random.default_rng(seed)
    is_cat = np.zeros(out.n_nodes, np.uint8)
    cat_left = np.zeros(out.n_nodes, np.uint64)
    full = (1 << n_categories) - 1
    for g in range(out.n_nodes):
        if out.left[g] >= 0 and int(out.feature[g]) in set(features):
            m = 0
            while m == 0 or m == full:
                m = int(sum(1 << c for c in range(n_categories) if rng.random() < 0.5))
            is_cat[g] = 1
            cat_left[g] = m
    out.is_cat, out.cat_left = is_cat, cat_left
    return out


def categorical_columns(X: np.ndarray, features, n_categories: int, seed: int,
                        other_frac: float = 0.1, nan_frac: float = 0.1) -> np.ndarray:
    """A copy of X whose `features` columns hold categories 0..n-1, with a
    fraction of values that are no category (negative, >= n, or >= 64) and a
    fraction of NaN."""
    out = np.array(X, dtype=np.float32, copy=True)
    rng = np.random.default_rng(seed)
    for f in features:
        col = rng.integers(0, n_categories, X.shape[0]).astype(np.float32)
        u = rng.random(X.shape[0])
        other = rng.choice(np.array([-1.0, -0.5, n_categories, n_categories + 0.5, 64.0, 1e6],
                                    dtype=np.float32), X.shape[0])
        col = np.where(u < other_frac, other, col)
        col = np.where((u >= other_frac) & (u < other_frac + nan_frac), np.nan, col)
        out[:, f] = col
    return out


def grow(seed: int, n_trees: int, max_depth: int, n_features: int, n_train: int,
         leaf_std: float, min_rows: int = 5, full_depth: bool = False) -> Ensemble:
    lib = _load()
    e = _Ens()
    rc = lib.synth_grow(seed, n_trees, max_depth, min_rows, int(full_depth), n_features, n_train,
                        leaf_std, _threads(), ctypes.byref(e))
    if rc != 0:
        raise RuntimeError(f"synth_grow failed ({rc})")
    try:
        n = e.n_nodes
        arr = lambda p, cnt: np.ctypeslib.as_array(p, shape=(cnt,)).copy()
        out = Ensemble(arr(e.node_offsets, n_trees + 1), arr(e.left, n), arr(e.right, n),
                       arr(e.feature, n), arr(e.threshold, n), arr(e.default_left, n),
                       arr(e.z, n), arr(e.leaf_value, n), arr(e.cover, n), n_features,
                       e.max_depth_seen)
    finally:
        lib.synth_free(ctypes.byref(e))
    return out


def normal(seed: int, stream: int, shape) -> np.ndarray:
    lib = _load()
    out = np.empty(shape, dtype=np.float32)
    lib.synth_normal_f32(seed, stream, out.size, _threads(), out.ctypes.data)
    return out


def uniform(seed: int, stream: int, ctr: int) -> float:
    return _load().synth_uniform(seed, stream, ctr)


def batch_draw(seed: int, n_ens: int = 64, trees=(10, 2000), depth=(3, 16), feats=(8, 200),
               samples=(1, 50000)):
    lib = _load()
    out = [np.zeros(n_ens, dtype=np.int32) for _ in range(4)]
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    lib.synth_batch_draw(seed, n_ens, trees[0], trees[1], depth[0], depth[1], feats[0], feats[1],
                         samples[0], samples[1], *[ptr(a) for a in out])
    return out  # trees, depth, n_features, n_samples


# --------------------------------------------------------------- workloads ---

# The fixed workloads, by name: (seed offset, shape).  The seed of each is
# SEED_BASE + its offset.
WORKLOADS = {
    # 10 trees grown to full depth 4, F = 8, M = 100: the small parity case
    "small-depth4": (0, dict(n_trees=10, max_depth=4, n_features=8, n_samples=100, n_train=1000,
                             leaf_std=1.0, full_depth=True)),
    # XGBoost-shaped: 1,000 trees of depth <= 8, F = 50, M = 10,000
    "xgb-depth8": (1, dict(n_trees=1000, max_depth=8, n_features=50, n_samples=10000, n_train=100000,
                           leaf_std=0.1, full_depth=False)),
    # deep unbalanced trees: 200 trees of depth <= 20 over F = 24 (repeated features), M = 5,000
    "deep-depth20": (2, dict(n_trees=200, max_depth=20, n_features=24, n_samples=5000, n_train=200000,
                             leaf_std=0.1, full_depth=False)),
    # pairwise interactions: 500 trees of depth <= 6, F = 30, M = 2,000
    "pairs-depth6": (3, dict(n_trees=500, max_depth=6, n_features=30, n_samples=2000, n_train=50000,
                             leaf_std=0.1, full_depth=False)),
}


class Workload:
    """One ensemble plus its sample matrix (and upstream gradient, if any)."""

    def __init__(self, name, ens: Ensemble, X: np.ndarray, grad_phi: np.ndarray | None = None,
                 meta: dict | None = None):
        self.name = name
        self.ens = ens
        self.X = X
        self.grad_phi = grad_phi
        self.meta = meta or {}

    @property
    def M(self) -> int:
        return self.X.shape[0]

    @property
    def F(self) -> int:
        return self.X.shape[1]


def workload(name: str, n_samples: int | None = None, n_trees: int | None = None,
             with_grad: bool = False) -> Workload:
    """One of the named fixed workloads, optionally with fewer samples or trees
    (the first trees and rows of the full workload: same seed and streams)."""
    off, shape = WORKLOADS[name]
    c = dict(shape)
    seed = SEED_BASE + off
    if n_trees is not None:
        c["n_trees"] = n_trees
    m = c["n_samples"] if n_samples is None else n_samples
    ens = grow(seed, c["n_trees"], c["max_depth"], c["n_features"], c["n_train"], c["leaf_std"],
               min_rows=5, full_depth=c["full_depth"])
    X = normal(seed, STREAM_X, (m, c["n_features"]))
    g = normal(seed, STREAM_GRAD, (m, c["n_features"] + 1)) if with_grad else None
    return Workload(name, ens, X, g, dict(c, seed=seed, n_samples=m))


def batch_config(n_ens: int = 64, seed: int | None = None, max_samples: int | None = None,
                 tree_scale: float = 1.0) -> list[Workload]:
    """The heterogeneous batch: n_ens ensembles with drawn sizes.  `max_samples`
    and `tree_scale` only shrink it for small test cases."""
    seed = SEED_BASE + 4 if seed is None else seed
    trees, depth, feats, samples = batch_draw(seed, n_ens)
    out = []
    for e in range(n_ens):
        es = seed * 1000 + e
        nt = max(1, int(round(trees[e] * tree_scale)))
        n_train = int(min(100000, 20 * 2 ** int(depth[e])))
        ens = grow(es, nt, int(depth[e]), int(feats[e]), n_train, 0.1, min_rows=5)
        m = int(samples[e]) if max_samples is None else int(min(samples[e], max_samples))
        X = normal(es, STREAM_X, (m, int(feats[e])))
        g = normal(es, STREAM_GRAD, (m, int(feats[e]) + 1))
        out.append(Workload(f"batch{e}", ens, X, g, dict(seed=es, n_trees=nt, depth=int(depth[e]),
                                                          n_features=int(feats[e]), n_samples=m,
                                                          n_train=n_train)))
    return out
