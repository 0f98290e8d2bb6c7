"""Shared test helpers: tiny ensembles (hand-written or seeded) and error norms."""
import json
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_trees():
    with open(os.path.join(GOLDEN, "hand_trees.json")) as fh:
        data = json.load(fh)
    out = []
    for t in data["trees"]:
        n = len(t["left"])
        ens = synth.Ensemble([0, n], t["left"], t["right"], t["feature"], t["threshold"],
                             t["default_left"], t["z"], t["leaf_value"], np.zeros(n), t["n_features"])
        out.append((t, ens))
    return out


def sample_x(s):
    return np.array([np.nan if v == "nan" else v for v in s["x"]], dtype=np.float32)


def tiny_ensemble(seed, n_trees=3, depth=5, F=6, n_train=200, full=False):
    """Seeded random-split ensemble; depth > F forces repeated features."""
    return synth.grow(seed, n_trees, depth, F, n_train, 1.0, min_rows=2, full_depth=full)


def rel_err_rows(phi, ref):
    """Per-sample error normalised by max(|f(x)|, max_i |phi_i|) of the reference:
    |f(x)| alone is fragile when the prediction is near zero."""
    fx = np.abs(ref.sum(axis=1))
    scale = np.maximum(fx, np.abs(ref[:, :-1]).max(axis=1))
    scale = np.maximum(scale, 1e-30)
    return np.abs(phi - ref).max(axis=1) / scale


def leaf_unique_counts(ens):
    """Per node: the number of distinct features split on along the root path
    of a leaf (its merged path length d), -1 at internal nodes."""
    out = np.full(ens.n_nodes, -1, dtype=np.int64)
    for t in range(ens.n_trees):
        base = int(ens.node_offsets[t])
        stack = [(0, frozenset())]
        while stack:
            v, feats = stack.pop()
            g = base + v
            if ens.left[g] < 0:
                out[g] = len(feats)
                continue
            nxt = feats | {int(ens.feature[g])}
            stack.append((int(ens.left[g]), nxt))
            stack.append((int(ens.right[g]), nxt))
    return out


def golden_categorical_trees():
    with open(os.path.join(GOLDEN, "categorical_trees.json")) as fh:
        data = json.load(fh)
    out = []
    for t in data["trees"]:
        n = len(t["left"])
        ens = synth.Ensemble([0, n], t["left"], t["right"], t["feature"], t["threshold"],
                             t["default_left"], t["z"], t["leaf_value"], np.zeros(n), t["n_features"],
                             is_cat=t["is_cat"], cat_left=t["cat_left"])
        out.append((t, ens))
    return out


def categorical_ensemble(seed, n_trees=3, depth=7, F=5, cat_features=(0, 2), n_categories=6,
                         n_train=500):
    """Seeded ensemble whose splits on `cat_features` are categorical (random
    left sets over n_categories), depth > F so features repeat on paths."""
    base = synth.grow(seed, n_trees, depth, F, n_train, 1.0, min_rows=2)
    return synth.make_categorical(base, cat_features, n_categories, seed + 1)


def caterpillar_ensemble(seed, depths, F):
    """One tree per entry of `depths`: every internal node has one leaf child
    and splits on a feature not used above it, so the longest path has
    `depth` unique features (the widest merged paths the library takes).
    Thresholds ~ N(0, 0.5), child weights w and 1 - w with w ~ U(0.2, 0.8),
    leaf values ~ N(0, 1), random default directions."""
    rng = np.random.default_rng(seed)
    parts = []
    for depth in depths:
        n = 2 * depth + 1
        left = np.full(n, -1, np.int32)
        right = np.full(n, -1, np.int32)
        feature = np.zeros(n, np.int32)
        thr = np.zeros(n, np.float32)
        z = np.ones(n, np.float32)
        val = np.zeros(n, np.float32)
        defl = rng.integers(0, 2, n).astype(np.uint8)
        feats = rng.permutation(F)[:depth]
        for k in range(depth):
            leaf = depth + 1 + k
            nxt = k + 1 if k + 1 < depth else depth  # the last internal node has two leaves
            a, b = (nxt, leaf) if rng.random() < 0.5 else (leaf, nxt)
            left[k], right[k] = a, b
            feature[k] = feats[k]
            thr[k] = rng.normal(0.0, 0.5)
            w = rng.uniform(0.2, 0.8)
            z[a], z[b] = w, 1.0 - w
        for v in range(n):
            if left[v] < 0:
                val[v] = rng.normal()
        parts.append(synth.Ensemble([0, n], left, right, feature, thr, defl, z, val, np.ones(n), F))
    return synth.concat(parts)
