"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every entry point the header declares, and its host preparation agrees with
the oracle's independent path walk."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
import paper_2605_04497_gb300 as qts
from helpers import golden_trees, tiny_ensemble

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_04497_gb300 import build as b

    b.build()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(qts_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol():
    declared = _declared()
    assert "qts_shap_values" in declared and "qts_load_ensemble" in declared
    L = ctypes.CDLL(qts.LIB_PATH)
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    assert set(qts.EXPORTS) <= declared


@pytest.mark.parametrize("n", [1, 2, 5, 8, 13, 16, 32])
def test_library_gauss_legendre_matches_oracle(n):
    """The library's Golub-Welsch/Jacobi rule against the oracle's Newton rule."""
    t, w = qts.gauss_legendre(n)
    to, wo = oracle.gl_nodes(n)
    assert np.allclose(t, to, atol=5e-15, rtol=0)
    assert np.allclose(w, wo, atol=5e-15, rtol=0)


def test_describe_matches_oracle_paths_and_bias():
    for seed, depth, F in [(3, 7, 5), (4, 10, 12), (5, 4, 30)]:
        ens = tiny_ensemble(seed, n_trees=5, depth=depth, F=F, n_train=3000)
        info = qts.describe(ens)
        n_paths, max_d, sum_d = oracle.path_stats(ens)
        assert info["n_paths"] == n_paths and info["max_unique"] == max_d
        assert info["sum_unique"] == sum_d
        assert sum(p for _, p in info["buckets"]) == n_paths
        phi = oracle.shap_exact(ens, np.zeros((1, F), np.float32))
        assert abs(info["expected_value"] - phi[0, F]) < 1e-12 * max(1, abs(phi[0, F]))


def test_describe_xgb_depth8_buckets():
    w = synth.workload("xgb-depth8", n_samples=1, n_trees=50)
    info = qts.describe(w.ens)
    widths = [d for d, _ in info["buckets"]]
    assert widths == sorted(widths) and max(widths) <= 8
    assert info["n_leaves"] == w.ens.n_leaves


def test_describe_rejects_bad_input():
    spec, ens = golden_trees()[0]
    bad = ens.copy()
    bad.left = bad.left.copy()
    bad.left[1] = 7  # child out of range
    with pytest.raises(qts.QtsError) as e:
        qts.describe(bad)
    assert e.value.status == 1
    bad = ens.copy()
    bad.z = bad.z.copy()
    bad.z[3] = 0.0  # edge weight must be > 0
    with pytest.raises(qts.QtsError) as e:
        qts.describe(bad)
    assert e.value.status == 1
    bad = ens.copy()
    bad.feature = bad.feature.copy()
    bad.feature[0] = 5  # feature out of range
    with pytest.raises(qts.QtsError):
        qts.describe(bad)


def test_describe_rejects_paths_beyond_64_unique_features():
    # a caterpillar tree splitting on 70 distinct features
    F, depth = 70, 70
    n = 2 * depth + 1
    left = -np.ones(n, np.int32)
    right = -np.ones(n, np.int32)
    feat = -np.ones(n, np.int32)
    for k in range(depth):
        node = 2 * k
        feat[node] = k
        left[node] = 2 * k + 2 if k + 1 < depth else 2 * k + 2
        right[node] = 2 * k + 1
    left[2 * (depth - 1)] = 2 * depth
    ens = synth.Ensemble([0, n], left, right, feat, np.zeros(n), np.zeros(n), np.full(n, 0.5, np.float32),
                         np.ones(n), np.zeros(n), F)
    with pytest.raises(qts.QtsError) as e:
        qts.describe(ens)
    assert e.value.status == 4


def test_triple_index_is_the_lexicographic_rank():
    """The compact third-order layout enumerates a < b < c in lexicographic order."""
    for F in (3, 4, 7, 12):
        idx = qts.triple_index(F)
        lex = [(a, b, c) for a in range(F) for b in range(a + 1, F) for c in range(b + 1, F)]
        assert [idx[t] for t in lex] == list(range(len(lex)))


def test_feature_with_both_split_types_is_rejected():
    """A feature is either numerical or categorical throughout an ensemble; the
    loader rejects a mix before touching the device."""
    from helpers import categorical_ensemble

    ens = categorical_ensemble(2300, n_trees=2, depth=5, F=3, cat_features=(0,))
    internal = np.flatnonzero((ens.left >= 0) & (ens.feature == 0))
    assert len(internal) >= 2
    ens.is_cat[internal[0]] = 0  # one numerical split on a categorical feature
    with pytest.raises(qts.QtsError) as ei:
        qts.Ensemble.from_arrays(ens)
    assert ei.value.status == 1 and "numerical and categorical" in str(ei.value)


# ------------------------------------------------ path tables, bit for bit

def _bucket_width(d):
    if d <= 16:
        return d
    for w in (20, 24, 28, 32, 40, 48, 56, 64):
        if d <= w:
            return w
    raise ValueError(d)


def _expected_tables(ens):
    """The merged paths written out from the tree arrays (Sec. 2, Eq. q_def):
    per leaf, the splits on each feature merged into one element with z the
    product of the edge weights (in FP64, rounded once), [lo, hi) the
    intersection of the numerical intervals, the intersection of the
    categorical sets, and NaN / other-value flags; elements sorted by feature,
    padded to the bucket width."""
    f32 = lambda v: int(np.float32(v).view(np.uint32))
    F = ens.n_features
    is_cat = getattr(ens, "is_cat", None)
    paths = []  # (width, tree order index, leaf, records)
    order = 0
    for t in range(ens.n_trees):
        base = int(ens.node_offsets[t])
        if ens.left[base] < 0:
            continue
        stack = [(0, [])]
        while stack:  # left subtree first
            v, edges = stack.pop()
            g = base + v
            if ens.left[g] >= 0:
                for side, c in ((1, int(ens.right[g])), (0, int(ens.left[g]))):
                    stack.append((c, edges + [(g, base + c, side == 0)]))
                continue
            elems = {}
            for (p, c, went_left) in edges:
                f = int(ens.feature[p])
                e = elems.setdefault(f, dict(z=1.0, lo=-np.inf, hi=np.inf, nan=True, cat=False,
                                             cats=(1 << 64) - 1, other=True))
                e["z"] *= float(ens.z[c])
                if is_cat is not None and is_cat[p]:
                    m = int(ens.cat_left[p])
                    e["cat"] = True
                    e["cats"] &= m if went_left else ((1 << 64) - 1) ^ m
                    if went_left:
                        e["other"] = False
                elif went_left:
                    e["hi"] = min(e["hi"], float(ens.threshold[p]))
                else:
                    e["lo"] = max(e["lo"], float(ens.threshold[p]))
                if went_left != bool(ens.default_left[p]):
                    e["nan"] = False
            d = len(elems)
            D = _bucket_width(d)
            zprod = 1.0
            recs = []
            for f in sorted(elems):
                e = elems[f]
                zprod *= e["z"]
                bits = f | (0x80000000 if e["nan"] else 0)
                if e["cat"]:
                    bits |= 0x40000000 | (0x20000000 if e["other"] else 0)
                    lo, hi = e["cats"] & 0xFFFFFFFF, e["cats"] >> 32
                else:
                    lo, hi = f32(e["lo"]), f32(e["hi"])
                recs.append([f32(e["z"]), lo, hi, bits])
            recs += [[f32(1.0), f32(-np.inf), f32(np.inf), F | 0x80000000]] * (D - d)
            head = [f32(float(ens.leaf_value[g])), f32(zprod), 0, 0]
            paths.append((D, order, g, [head] + recs))
            order += 1
    paths.sort(key=lambda p: (p[0], p[1]))
    rec = np.array([r for p in paths for r in p[3]], dtype=np.uint64).reshape(-1, 4).astype(np.uint32)
    return rec, np.array([p[2] for p in paths], dtype=np.int64), np.array([p[0] for p in paths], dtype=np.int32)


@pytest.mark.parametrize("case", ["repeated", "wide", "categorical"])
def test_path_tables_bit_for_bit(case):
    """The library's prepared tables equal the merged paths written out in
    Python from the tree arrays, bit for bit (row a1 of the hot path)."""
    from helpers import caterpillar_ensemble, categorical_ensemble

    if case == "repeated":
        ens = tiny_ensemble(3300, n_trees=5, depth=11, F=5, n_train=3000)
        rng = np.random.default_rng(3300)
        ens.default_left[:] = rng.integers(0, 2, ens.n_nodes).astype(np.uint8)
    elif case == "wide":
        ens = caterpillar_ensemble(3301, (3, 18, 33, 62), 64)
    else:
        ens = categorical_ensemble(3302, n_trees=4, depth=9, F=5, cat_features=(0, 3))
    got = qts.describe_paths(ens)
    rec, leaf, width = _expected_tables(ens)
    assert np.array_equal(got["path_leaf"], leaf)
    assert np.array_equal(got["path_width"], width)
    assert got["records"].shape == rec.shape
    assert np.array_equal(got["records"], rec)
    if case == "categorical":
        assert (rec[:, 3] & 0x40000000).any() and ((rec[:, 3] & 0x60000000) == 0x60000000).any()
    if case == "wide":
        assert set(width) >= {3, 20, 40, 64}
    if case == "repeated":
        assert not ((rec[:, 3] & 0x80000000) != 0).all()  # some merged elements reject NaN


def test_host_rejects_malformed_models():
    """Bad input is refused on the host with an error code before any device
    work: too many features, a NaN threshold, a non-finite leaf value, a node
    reached twice, a self-loop, offsets that do not increase."""
    spec, ens = golden_trees()[0]

    def expect(bad, status, fn=qts.describe):
        with pytest.raises(qts.QtsError) as e:
            fn(bad)
        assert e.value.status == status, (e.value.status, str(e.value))

    big = ens.copy()
    big.n_features = 833  # one above QTS_MAX_FEATURES
    expect(big, 4)
    expect(big, 4, qts.describe_paths)
    bad = ens.copy()
    bad.threshold[0] = np.nan
    expect(bad, 1)
    bad = ens.copy()
    bad.leaf_value[2] = np.inf
    expect(bad, 1, qts.describe_paths)
    # node 1 reached from the root and from node 1 itself
    bad = ens.copy()
    bad.left[1], bad.right[1] = 3, 1
    expect(bad, 1)
    # two parents share a child: node 3 hangs below node 0 and node 1
    bad = ens.copy()
    bad.right[0] = 3
    expect(bad, 1)
    bad = ens.copy()
    bad.node_offsets = np.array([0, 5, 5], np.int64)
    expect(bad, 1)


def _expected_alg1_program(ens):
    """Algorithm 1's per-node data written out from the tree arrays: internal
    nodes in preorder, the merged z of the node's feature before it and through
    each child edge (FP64 products, rounded once), the nearest ancestor on the
    same feature, leaf flags and values."""
    f32 = lambda v: int(np.float32(v).view(np.uint32))
    recs, off, deepest = [], [0], -1
    for t in range(ens.n_trees):
        base = int(ens.node_offsets[t])

        def visit(v, depth, zcur, anc):
            nonlocal deepest
            g = base + v
            deepest = max(deepest, depth)
            f = int(ens.feature[g])
            ch = (int(ens.left[g]), int(ens.right[g]))
            zold = zcur.get(f, 1.0)
            leaf = [ens.left[base + c] < 0 for c in ch]
            meta = f | (anc.get(f, 127) << 16) | (int(leaf[0]) << 23) | (int(leaf[1]) << 24) | \
                (int(ens.default_left[g] != 0) << 25)
            recs.append([f32(ens.threshold[g]), f32(zold * float(ens.z[base + ch[0]])),
                         f32(zold * float(ens.z[base + ch[1]])), f32(zold),
                         f32(ens.leaf_value[base + ch[0]] if leaf[0] else 0.0),
                         f32(ens.leaf_value[base + ch[1]] if leaf[1] else 0.0), meta, depth])
            for i, c in enumerate(ch):
                if not leaf[i]:
                    visit(c, depth + 1, {**zcur, f: zold * float(ens.z[base + c])}, {**anc, f: depth})

        if ens.left[base] >= 0:
            visit(0, 0, {}, {})
        off.append(len(recs))
    return np.array(recs, dtype=np.uint64).astype(np.uint32), np.array(off), deepest + 1


def test_alg1_program_bit_for_bit():
    """The depth-first form's record program equals the per-node data written
    out in Python from the tree arrays, bit for bit, on trees with repeated
    features and random default directions plus a single-leaf tree."""
    base = tiny_ensemble(3400, n_trees=4, depth=12, F=4, n_train=3000)
    rng = np.random.default_rng(3400)
    base.default_left[:] = rng.integers(0, 2, base.n_nodes).astype(np.uint8)
    stump = synth.Ensemble([0, 1], [-1], [-1], [0], [0.0], [1], [1.0], [2.5], [1], 4)
    ens = synth.concat([base, stump, base.tree(2)])
    got = qts.describe_alg1_program(ens)
    rec, off, levels = _expected_alg1_program(ens)
    assert np.array_equal(got["tree_off"], off)
    assert got["levels"] == levels
    assert np.array_equal(got["records"], rec)
    assert ((rec[:, 6] >> 16) & 127 != 127).any()  # repeated features occur


def _pair_count(ens):
    """Sibling pairs (internal nodes whose two children are leaves) and the sum
    of their merged path lengths: the features on the way to the node plus the
    node's own feature."""
    n = sd = 0
    for t in range(ens.n_trees):
        base = int(ens.node_offsets[t])
        stack = [(0, frozenset())]
        while stack:
            v, fs = stack.pop()
            g = base + v
            if ens.left[g] < 0:
                continue
            l, r = base + int(ens.left[g]), base + int(ens.right[g])
            f = int(ens.feature[g])
            if ens.left[l] < 0 and ens.left[r] < 0:
                n += 1
                sd += len(fs | {f})
                continue
            stack.append((int(ens.left[g]), fs | {f}))
            stack.append((int(ens.right[g]), fs | {f}))
    return n, sd


@pytest.mark.parametrize("seed,depth,F", [(61, 6, 9), (62, 12, 5), (63, 4, 3), (64, 9, 40)])
def test_pair_tables_count_and_bias(seed, depth, F):
    """The batched pass's tables hold each sibling pair as one path: one path
    fewer per pair, the pair's merged length counted once, every leaf kept, and
    the same E[f] (the pair element's z is val_A z_A + val_B z_B)."""
    ens = synth.grow(seed, 7, depth, F, 3000, 1.0, min_rows=2)
    full = qts.describe(ens)
    pairs = qts.describe(ens, pairs=True)
    n_pairs, sd_pairs = _pair_count(ens)
    assert n_pairs > 0
    assert pairs["n_leaves"] == full["n_leaves"]
    assert pairs["n_paths"] == full["n_paths"] - n_pairs
    assert pairs["sum_unique"] == full["sum_unique"] - sd_pairs
    assert pairs["expected_value"] == pytest.approx(full["expected_value"], rel=1e-12, abs=1e-12)
