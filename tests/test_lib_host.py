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
