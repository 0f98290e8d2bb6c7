"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Each test pins one oracle function to something other than itself: hand-derived
values (tests/golden), closed forms, the Shapley axioms, a library quadrature
routine, brute-force subset enumeration, or finite differences.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import golden_trees, rel_err_rows, sample_x, tiny_ensemble


# ------------------------------------------------------------ Gauss-Legendre

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 16, 24, 32])
def test_gl_exact_on_monomials(n):
    """n-point Gauss-Legendre integrates t^k exactly for k <= 2n-1 (Sec. 4, Thm 2)."""
    t, w = oracle.gl_nodes(n)
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < 1
    assert abs(w.sum() - 1.0) < 1e-14
    for k in range(2 * n):
        assert abs((w * t**k).sum() - 1.0 / (k + 1)) < 1e-14, k
    # degree 2n: the rule's remainder for t^(2n) on [0,1] is (n!)^4 / ((2n+1) ((2n)!)^2)
    if n <= 8:
        rem = math.factorial(n) ** 4 / ((2 * n + 1) * math.factorial(2 * n) ** 2)
        got = 1.0 / (2 * n + 1) - (w * t ** (2 * n)).sum()
        assert abs(got - rem) < 1e-9 * rem + 1e-16, (got, rem)


@pytest.mark.parametrize("n", [1, 4, 8, 20])
def test_gl_matches_numpy_leggauss(n):
    """Same nodes as numpy's independent Golub-Welsch implementation, mapped to [0,1]."""
    x, wx = np.polynomial.legendre.leggauss(n)
    t, w = oracle.gl_nodes(n)
    assert np.allclose(t, (x + 1) / 2, atol=1e-14)
    assert np.allclose(w, wx / 2, atol=1e-14)


def test_gl_closed_forms():
    t, w = oracle.gl_nodes(1)
    assert t[0] == 0.5 and w[0] == 1.0
    t, w = oracle.gl_nodes(2)
    r = 1 / (2 * math.sqrt(3))
    assert np.allclose(t, [0.5 - r, 0.5 + r], atol=1e-15) and np.allclose(w, [0.5, 0.5], atol=1e-15)


# ------------------------------------------------------------ hand-derived

def test_golden_hand_trees():
    """Every formulation reproduces the values derived by hand in tests/golden."""
    for spec, ens in golden_trees():
        for s in spec["samples"]:
            x = sample_x(s)
            want = np.array(s["phi"])
            bf_phi, bf_sii = oracle.brute_force(ens, x)
            ex = oracle.shap_exact(ens, x[None])[0]
            a1 = oracle.alg1(ens, x, 1, 8)
            sii, _ = oracle.sii_exact(ens, x[None])
            a2 = oracle.alg1(ens, x, 2, 8)
            for got in (bf_phi, ex, a1):
                assert np.allclose(got, want, atol=1e-15, rtol=0), (spec["name"], got, want)
            for got in (bf_sii[0, 1], sii[0, 0, 1], a2[0, 1]):
                assert abs(got - s["sii01"]) < 1e-15, (spec["name"], got)
            assert abs(oracle.predict(ens, x[None])[0] - s["fx"]) == 0
            if "sii012" in s:
                for got in (oracle.brute_force3(ens, x)[0, 1, 2], oracle.sii3_exact(ens, x[None])[0, 0, 1, 2],
                            oracle.alg1(ens, x, 3, 8)[2, 0, 1]):
                    assert abs(got - s["sii012"]) < 1e-15, (spec["name"], got)


def test_stump_closed_form():
    """Single split on feature i: phi_i = val_taken - (w_l val_l + w_r val_r), others 0."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        F = 5
        i = int(rng.integers(F))
        cl, cr = rng.integers(1, 100, size=2)
        vl, vr = rng.standard_normal(2).astype(np.float32)
        thr = np.float32(rng.standard_normal())
        zl, zr = np.float32(cl / (cl + cr)), np.float32(cr / (cl + cr))
        ens = synth.Ensemble([0, 3], [1, -1, -1], [2, -1, -1], [i, -1, -1], [thr, 0, 0], [0, 0, 0],
                             [1, zl, zr], [0, vl, vr], [0, 0, 0], F)
        x = rng.standard_normal(F).astype(np.float32)
        taken = vl if x[i] < thr else vr
        ef = float(zl) * float(vl) + float(zr) * float(vr)
        phi = oracle.shap_exact(ens, x[None])[0]
        want = np.zeros(F + 1)
        want[i] = float(taken) - ef
        want[F] = ef
        assert np.allclose(phi, want, atol=1e-15)


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("seed", range(12))
def test_exact_equals_brute_force(seed):
    """Exact Bernstein expansion of Thm 1 == subset enumeration of the game,
    including repeated features on a path (depth 7 > F = 5)."""
    ens = tiny_ensemble(1000 + seed, n_trees=3, depth=7, F=5)
    X = synth.normal(77 + seed, 1, (4, 5))
    phi = oracle.shap_exact(ens, X)
    sii, _ = oracle.sii_exact(ens, X)
    for s in range(X.shape[0]):
        bf_phi, bf_sii = oracle.brute_force(ens, X[s])
        scale = max(1.0, np.abs(bf_phi).max())
        assert np.abs(phi[s] - bf_phi).max() < 1e-12 * scale
        assert np.abs(sii[s] - bf_sii).max() < 1e-12 * scale


def test_null_player_and_player_count():
    """Adding never-split features leaves phi unchanged and gives them exactly
    zero (Sec. 2 null player; Lemma 2 case 1) -- brute force over F and F+3."""
    ens = tiny_ensemble(5, n_trees=2, depth=4, F=4)
    X = synth.normal(5, 2, (3, 4))
    big = ens.copy()
    big.n_features = 7
    Xb = np.concatenate([X, synth.normal(5, 3, (3, 3))], axis=1)
    for s in range(3):
        a, _ = oracle.brute_force(ens, X[s])
        b, _ = oracle.brute_force(big, Xb[s])
        assert np.allclose(a[:4], b[:4], atol=1e-13)
        assert np.abs(b[4:7]).max() < 1e-13
        assert abs(a[4] - b[7]) < 1e-13
        c = oracle.shap_exact(big, Xb[s:s + 1])[0]
        assert np.all(c[4:7] == 0.0)


# ------------------------------------------------------------ axioms

def test_efficiency_local_accuracy():
    """sum_i phi_i + E[f] = f(x) (the paper's accuracy metric, Sec. 8)."""
    w = synth.workload("small-depth4")
    phi = oracle.shap_exact(w.ens, w.X)
    f = oracle.predict(w.ens, w.X)
    assert np.abs(phi.sum(axis=1) - f).max() < 1e-12
    sub = synth.workload("xgb-depth8", n_samples=20, n_trees=20)
    phi = oracle.shap_exact(sub.ens, sub.X)
    f = oracle.predict(sub.ens, sub.X)
    assert np.abs(phi.sum(axis=1) - f).max() < 1e-12


def test_symmetry_under_feature_relabelling():
    ens = tiny_ensemble(11, n_trees=3, depth=5, F=6)
    X = synth.normal(11, 1, (5, 6))
    perm = np.array([3, 0, 5, 1, 4, 2])  # new label of old feature k is perm[k]
    rel = ens.copy()
    rel.feature = np.where(ens.feature >= 0, perm[np.maximum(ens.feature, 0)], -1).astype(np.int32)
    Xr = np.empty_like(X)
    Xr[:, perm] = X
    a = oracle.shap_exact(ens, X)
    b = oracle.shap_exact(rel, Xr)
    assert np.allclose(b[:, perm], a[:, :6], atol=1e-14)
    assert np.allclose(a[:, 6], b[:, 6], atol=1e-14)


def test_linearity_in_trees_and_leaf_values():
    ens = tiny_ensemble(21, n_trees=4, depth=5, F=6)
    X = synth.normal(21, 1, (6, 6))
    whole = oracle.shap_exact(ens, X)
    parts = sum(oracle.shap_exact(ens.tree(t), X) for t in range(ens.n_trees))
    assert np.allclose(whole, parts, atol=1e-13)
    scaled = ens.copy()
    scaled.leaf_value = (ens.leaf_value * np.float32(2.0)).astype(np.float32)
    assert np.allclose(oracle.shap_exact(scaled, X), 2.0 * whole, atol=1e-13)


def test_missing_values_follow_default_direction():
    ens = tiny_ensemble(31, n_trees=3, depth=5, F=5)
    X = synth.normal(31, 1, (6, 5))
    X[0, 1] = np.nan
    X[1, :] = np.nan
    X[2, 3] = np.nan
    phi = oracle.shap_exact(ens, X)
    f = oracle.predict(ens, X)
    assert np.abs(phi.sum(axis=1) - f).max() < 1e-12
    for s in range(3):
        bf, _ = oracle.brute_force(ens, X[s])
        assert np.allclose(phi[s], bf, atol=1e-12)


# ------------------------------------------------------------ interactions

def test_interaction_matrix_properties():
    """Rows of the pred_interactions layout sum to phi_i; the whole matrix sums
    to f(x); off-diagonal entries are SII/2 and symmetric."""
    w = synth.workload("pairs-depth6", n_samples=8, n_trees=10)
    sii, phi = oracle.sii_exact(w.ens, w.X)
    mat = oracle.interaction_matrix(sii, phi)
    F = w.F
    assert np.allclose(mat[:, :F, :F].sum(axis=2), phi[:, :F], atol=1e-13)
    assert np.allclose(mat.sum(axis=(1, 2)), oracle.predict(w.ens, w.X), atol=1e-12)
    assert np.allclose(mat, np.transpose(mat, (0, 2, 1)), atol=0)


# ------------------------------------------------------------ Algorithm 1 / Thm 2

@pytest.mark.parametrize("order", [1, 2])
def test_alg1_exact_at_theorem2_bound(order):
    """Alg. 1 with n = ceil((d - s + 1)/2) points is exact (Thm 2)."""
    ens = tiny_ensemble(41, n_trees=3, depth=9, F=9, n_train=2000)
    _, dmax, _ = oracle.path_stats(ens)
    X = synth.normal(41, 1, (3, 9))
    n = math.ceil((dmax - order + 1) / 2)
    for s in range(3):
        if order == 1:
            ref = oracle.shap_exact(ens, X[s:s + 1])[0]
        else:
            ref = oracle.sii_exact(ens, X[s:s + 1], with_phi=False)[0][0]
        got = oracle.alg1(ens, X[s], order, n)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(got - ref).max() < 1e-12 * scale


def test_alg1_threaded_equals_single_sample_dfs_and_exact():
    """The threaded Algorithm 1 runs the same DFS per row (bit-identical to
    the single-sample call, whatever the thread count) and, with 8 points on
    paths of at most 16 unique features, equals the exact expansion (Thm 2)."""
    sub = synth.workload("xgb-depth8", n_samples=9, n_trees=12)
    a = oracle.alg1_shap(sub.ens, sub.X, 8, n_threads=4)
    b = oracle.alg1_shap(sub.ens, sub.X, 8, n_threads=1)
    assert np.array_equal(a, b)
    for s in range(sub.X.shape[0]):
        assert np.array_equal(a[s], oracle.alg1(sub.ens, sub.X[s], 1, 8))
    ref = oracle.shap_exact(sub.ens, sub.X)
    assert rel_err_rows(a, ref).max() < 1e-12
    assert oracle.alg1_shap(sub.ens, sub.X[:0], 8).shape == (0, sub.F + 1)


def test_quadrature_exact_iff_degree_covered():
    """n-point quadrature equals the exact integral for paths with d <= 2n
    unique features (integrand degree d - 1 <= 2n - 1), and misses it once d
    exceeds 2n."""
    ens = tiny_ensemble(51, n_trees=4, depth=10, F=10, n_train=4000)
    _, dmax, _ = oracle.path_stats(ens)
    assert dmax >= 8
    X = synth.normal(51, 1, (4, 10))
    ref = oracle.shap_exact(ens, X)
    ok = oracle.shap_quad(ens, X, math.ceil(dmax / 2))
    assert np.abs(ok - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    low = oracle.shap_quad(ens, X, 2)
    assert np.abs(low - ref).max() > 1e-9


def test_eight_points_exact_on_depth8_config():
    sub = synth.workload("xgb-depth8", n_samples=10, n_trees=30)
    ref = oracle.shap_exact(sub.ens, sub.X)
    q = oracle.shap_quad(sub.ens, sub.X, 8)
    assert rel_err_rows(q, ref).max() < 1e-13


# ------------------------------------------------------------ gradients

def _loss_brute(ens, X, G):
    tot = 0.0
    for s in range(X.shape[0]):
        phi, _ = oracle.brute_force(ens, X[s])
        tot += float((G[s].astype(np.float64) * phi).sum())
    return tot


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_finite_differences_of_brute_force(seed):
    """phi is linear in every leaf value and every single edge weight, so a
    central difference of the brute-force game is exact up to rounding."""
    ens = tiny_ensemble(61 + seed, n_trees=2, depth=5, F=4, n_train=100)
    X = synth.normal(61 + seed, 1, (5, 4))
    G = synth.normal(61 + seed, 2, (5, 5))
    d_leaf, d_z = oracle.grad_exact(ens, X, G)
    roots = set(int(o) for o in ens.node_offsets[:-1])
    for n in range(ens.n_nodes):
        for name, g in (("leaf_value", d_leaf), ("z", d_z)):
            if name == "leaf_value" and ens.left[n] >= 0:
                assert g[n] == 0.0
                continue
            if name == "z" and n in roots:
                continue
            h = 1.0 if name == "leaf_value" else 1e-2
            ep, em = ens.copy(), ens.copy()
            getattr(ep, name)[n] += np.float32(h)
            getattr(em, name)[n] -= np.float32(h)
            hp = float(getattr(ep, name)[n]) - float(getattr(em, name)[n])
            fd = (_loss_brute(ep, X, G) - _loss_brute(em, X, G)) / hp
            assert abs(fd - g[n]) <= 1e-10 * max(1.0, abs(g[n])), (name, n, fd, g[n])


def test_gradient_leaf_subset_is_exact_at_listed_leaves():
    ens = tiny_ensemble(71, n_trees=3, depth=5, F=5)
    X = synth.normal(71, 1, (7, 5))
    G = synth.normal(71, 2, (7, 6))
    full_l, full_z = oracle.grad_exact(ens, X, G)
    leaves = np.flatnonzero(ens.left < 0)[::3]
    # global leaf index -> local within tree: grad_exact takes global node indices
    sub_l, sub_z = oracle.grad_exact(ens, X, G, leaves=leaves)
    assert np.allclose(sub_l[leaves], full_l[leaves], atol=1e-13)
    assert np.allclose(sub_z[leaves], full_z[leaves], atol=1e-13)


def test_threads_do_not_change_results():
    w = synth.workload("small-depth4")
    a = oracle.shap_exact(w.ens, w.X, n_threads=1)
    b = oracle.shap_exact(w.ens, w.X, n_threads=7)
    assert np.array_equal(a, b)


# ------------------------------------------------------------ third order

@pytest.mark.parametrize("seed", range(6))
def test_third_order_exact_equals_brute_force(seed):
    """Thm 1 with |S| = 3 integrated exactly == subset enumeration with the
    order-3 Shapley interaction weights (App. C), repeated features included."""
    ens = tiny_ensemble(1600 + seed, n_trees=3, depth=8, F=6)
    X = synth.normal(1600 + seed, 1, (3, 6))
    s3 = oracle.sii3_exact(ens, X)
    for s in range(3):
        bf = oracle.brute_force3(ens, X[s])
        assert np.abs(s3[s] - bf).max() < 1e-12 * max(1.0, np.abs(bf).max())
        assert np.allclose(bf, np.transpose(bf, (1, 0, 2)), atol=0)
        assert np.allclose(bf, np.transpose(bf, (0, 2, 1)), atol=0)


def test_third_order_alg1_exact_at_theorem2_bound():
    """Algorithm 1 with s = 3 and n = ceil((d - 2)/2) points is exact (Thm 2)."""
    ens = tiny_ensemble(1700, n_trees=3, depth=10, F=9, n_train=3000)
    _, dmax, _ = oracle.path_stats(ens)
    X = synth.normal(1700, 1, (2, 9))
    n = math.ceil((dmax - 3 + 1) / 2)
    ref = oracle.sii3_exact(ens, X)
    for s in range(2):
        got = oracle.alg1(ens, X[s], 3, n)
        assert np.abs(got - ref[s]).max() < 1e-12 * max(1.0, np.abs(ref[s]).max())


# ------------------------------------------------------------ categorical splits

def test_golden_categorical_trees():
    """Hand-derived values with categorical splits: a stump (category in the
    set, a fractional value, values that are no category, NaN) and a feature
    whose two categorical splits intersect along a path."""
    from helpers import golden_categorical_trees

    for spec, ens in golden_categorical_trees():
        for s in spec["samples"]:
            x = sample_x(s)
            want = np.array(s["phi"])
            bf_phi, _ = oracle.brute_force(ens, x)
            ex = oracle.shap_exact(ens, x[None])[0]
            a1 = oracle.alg1(ens, x, 1, 8)
            for got in (bf_phi, ex, a1):
                assert np.allclose(got, want, atol=1e-15, rtol=0), (spec["name"], s["x"], got, want)
            assert oracle.predict(ens, x[None])[0] == s["fx"]


@pytest.mark.parametrize("seed", range(5))
def test_categorical_exact_equals_brute_force(seed):
    """The merged category sets of the exact expansion against subset
    enumeration of the game, which follows each categorical split on its own;
    inputs include values that are no category and NaN."""
    from helpers import categorical_ensemble

    ens = categorical_ensemble(1700 + seed, n_trees=2, depth=7, F=5)
    X = synth.categorical_columns(synth.normal(1700 + seed, 1, (6, 5)), (0, 2), 6, 1700 + seed)
    ex_sii, ex_phi = oracle.sii_exact(ens, X)
    for s in range(X.shape[0]):
        bf_phi, bf_sii = oracle.brute_force(ens, X[s])
        assert np.allclose(ex_phi[s], bf_phi, atol=1e-13, rtol=0)
        assert np.allclose(ex_sii[s], bf_sii, atol=1e-13, rtol=0)
    assert np.allclose(ex_phi.sum(axis=1), oracle.predict(ens, X), atol=1e-12)
    a1 = np.stack([oracle.alg1(ens, X[s], 1, 8) for s in range(X.shape[0])])
    assert np.allclose(a1, ex_phi, atol=1e-12)


# ------------------------------------------------------------ any order

def _dense_to_compact(dense, F, s):
    import itertools

    return np.array([dense[c] for c in itertools.combinations(range(F), s)])


@pytest.mark.parametrize("seed", range(3))
def test_any_order_exact_equals_brute_force(seed):
    """Thm 1 with |S| = s integrated exactly against subset enumeration with the
    order-s weights of App. C, s = 1..6, repeated features included; the
    brute force writes subsets in enumeration order and the expansion by the
    rank formula, so agreement also pins the compact layout."""
    ens = tiny_ensemble(2400 + seed, n_trees=3, depth=9, F=7, n_train=3000)
    X = synth.normal(2400 + seed, 1, (3, 7))
    for s in range(1, 7):
        ex = oracle.sii_order_exact(ens, X, s)
        for r in range(X.shape[0]):
            bf = oracle.brute_force_order(ens, X[r], s)
            scale = max(1.0, np.abs(bf).max())
            assert np.abs(ex[r] - bf).max() < 1e-12 * scale, (s, r)


def test_any_order_reduces_to_orders_one_to_three():
    ens = tiny_ensemble(2450, n_trees=3, depth=8, F=6, n_train=2000)
    X = synth.normal(2450, 1, (4, 6))
    phi = oracle.shap_exact(ens, X)
    sii2, _ = oracle.sii_exact(ens, X)
    sii3 = oracle.sii3_exact(ens, X)
    o1 = oracle.sii_order_exact(ens, X, 1)
    o2 = oracle.sii_order_exact(ens, X, 2)
    o3 = oracle.sii_order_exact(ens, X, 3)
    for r in range(4):
        assert np.allclose(o1[r], phi[r, :6], atol=1e-14)
        assert np.allclose(o2[r], _dense_to_compact(sii2[r], 6, 2), atol=1e-14)
        assert np.allclose(o3[r], _dense_to_compact(sii3[r], 6, 3), atol=1e-14)


@pytest.mark.parametrize("s", [4, 5])
def test_any_order_alg1_exact_at_theorem2_bound(s):
    """Algorithm 1 of order s with n = ceil((d - s + 1)/2) points is exact (Thm 2)."""
    ens = tiny_ensemble(2500 + s, n_trees=3, depth=10, F=8, n_train=4000)
    _, dmax, _ = oracle.path_stats(ens)
    X = synth.normal(2500 + s, 1, (3, 8))
    n = max(1, math.ceil((dmax - s + 1) / 2))
    ref = oracle.sii_order_exact(ens, X, s)
    for r in range(3):
        got = oracle.alg1_order(ens, X[r], s, n)
        assert np.abs(got - ref[r]).max() < 1e-12 * max(1.0, np.abs(ref[r]).max())


def test_any_order_golden_chain():
    """The hand-derived third-order value of the three-feature chain, and the
    closed form for s = d: a path whose every feature is in S contributes
    val prod (o_i - z_i) (the integral of the empty product is 1)."""
    spec, ens = [g for g in golden_trees() if g[0]["name"] == "three_feature_chain"][0]
    x = sample_x(spec["samples"][0])
    for fn in (lambda: oracle.sii_order_exact(ens, x[None], 3)[0], lambda: oracle.brute_force_order(ens, x, 3),
               lambda: oracle.alg1_order(ens, x, 3, 8)):
        assert abs(fn()[0] - spec["samples"][0]["sii012"]) < 1e-15


@pytest.mark.parametrize("s", [4, 5, 6])
def test_any_order_closed_form_on_a_caterpillar(s):
    """A caterpillar tree of depth s (one leaf child per internal node, a new
    feature at every level): only its two deepest leaves use all s features, so
    SII over those features is the integral of an empty product (= 1) times
    val prod_i (o_i - z_i) summed over those two leaves (Thm 1), computed here
    from the tree arrays."""
    from helpers import caterpillar_ensemble

    ens = caterpillar_ensemble(3200 + s, [s], s + 2)
    X = synth.normal(3200 + s, 1, (5, s + 2))
    feats = sorted(int(f) for f in ens.feature[:s])
    import itertools

    rank = list(itertools.combinations(range(s + 2), s)).index(tuple(feats))
    for r in range(X.shape[0]):
        x = X[r]
        want = 0.0
        for leaf in (v for v in range(ens.n_nodes) if ens.left[v] < 0):
            # walk down from the root to this leaf, collecting (o - z) per level
            path, v, ok = [], 0, False
            while ens.left[v] >= 0:
                for c in (int(ens.left[v]), int(ens.right[v])):
                    if c == leaf or (ens.left[c] >= 0 and _reaches(ens, c, leaf)):
                        goes_left = c == ens.left[v]
                        o = float((x[ens.feature[v]] < ens.threshold[v]) == goes_left)
                        path.append(o - float(ens.z[c]))
                        v = c
                        break
            if len(path) == s:
                want += float(ens.leaf_value[leaf]) * float(np.prod(path))
        got = (oracle.sii_order_exact(ens, x[None], s)[0][rank], oracle.brute_force_order(ens, x, s)[rank],
               oracle.alg1_order(ens, x, s, 8)[rank])
        for g in got:
            assert abs(g - want) < 1e-13 * max(1.0, abs(want)), (s, r, g, want)


def _reaches(ens, v, target):
    if v == target:
        return True
    if ens.left[v] < 0:
        return False
    return _reaches(ens, int(ens.left[v]), target) or _reaches(ens, int(ens.right[v]), target)


def test_categorical_gradient_matches_finite_differences():
    """The analytic gradient with categorical splits against central
    differences of the brute force (phi is linear in each leaf value and each
    edge weight, so the difference is exact to rounding)."""
    from helpers import categorical_ensemble

    ens = categorical_ensemble(3500, n_trees=2, depth=5, F=3, cat_features=(0,), n_categories=5)
    X = synth.categorical_columns(synth.normal(3500, 1, (5, 3)), (0,), 5, 3500)
    G = synth.normal(3500, 2, (5, 4))
    d_leaf, d_z = oracle.grad_exact(ens, X, G)
    roots = set(int(o) for o in ens.node_offsets[:-1])
    checked = 0
    for n in range(ens.n_nodes):
        for name, g in (("leaf_value", d_leaf), ("z", d_z)):
            if (name == "leaf_value" and ens.left[n] >= 0) or (name == "z" and n in roots):
                continue
            h = 1.0 if name == "leaf_value" else 1e-2
            ep, em = ens.copy(), ens.copy()
            getattr(ep, name)[n] += np.float32(h)
            getattr(em, name)[n] -= np.float32(h)
            hp = float(getattr(ep, name)[n]) - float(getattr(em, name)[n])
            fd = (_loss_brute(ep, X, G) - _loss_brute(em, X, G)) / hp
            assert abs(fd - g[n]) <= 1e-10 * max(1.0, abs(g[n])), (name, n, fd, g[n])
            checked += 1
    assert checked > 20


@pytest.mark.parametrize("s", [3, 4])
def test_any_order_categorical_exact_equals_brute_force(s):
    from helpers import categorical_ensemble

    ens = categorical_ensemble(3600 + s, n_trees=2, depth=8, F=6, cat_features=(1, 4))
    X = synth.categorical_columns(synth.normal(3600 + s, 1, (4, 6)), (1, 4), 6, 3600 + s)
    ex = oracle.sii_order_exact(ens, X, s)
    for r in range(X.shape[0]):
        bf = oracle.brute_force_order(ens, X[r], s)
        assert np.abs(ex[r] - bf).max() < 1e-12 * max(1.0, np.abs(bf).max()), (s, r)
        a1 = oracle.alg1_order(ens, X[r], s, 8)
        assert np.abs(a1 - bf).max() < 1e-12 * max(1.0, np.abs(bf).max()), (s, r)
