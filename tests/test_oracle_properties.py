"""Randomised properties of the FP64 oracle (hypothesis; skipped where the
package is missing).  Each example draws a tiny seeded ensemble, optionally
with categorical splits, and inputs with NaN and non-category values, then
checks the exact expansion against subset enumeration of the game (Shapley
values and pairwise indices), local accuracy, and null players."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


@settings(max_examples=40, deadline=None, derandomize=True, database=None)
@given(seed=st.integers(0, 10**6), F=st.integers(2, 7), depth=st.integers(1, 9), n_trees=st.integers(1, 3),
       categorical=st.booleans(), nan_frac=st.sampled_from([0.0, 0.2]))
def test_exact_expansion_against_brute_force(seed, F, depth, n_trees, categorical, nan_frac):
    ens = synth.grow(seed, n_trees, depth, F, 400, 1.0, min_rows=2)
    X = synth.normal(seed, 1, (3, F))
    if categorical:
        cat = (0,)
        ens = synth.make_categorical(ens, cat, 5, seed + 7)
        X = synth.categorical_columns(X, cat, 5, seed + 11)
    rng = np.random.default_rng(seed)
    X[rng.random(X.shape) < nan_frac] = np.nan
    sii, phi = oracle.sii_exact(ens, X)
    fx = oracle.predict(ens, X)
    used = set(int(f) for f in ens.feature[ens.left >= 0])
    for r in range(X.shape[0]):
        bf_phi, bf_sii = oracle.brute_force(ens, X[r])
        scale = max(1.0, np.abs(bf_phi).max())
        assert np.abs(phi[r] - bf_phi).max() < 1e-12 * scale
        assert np.abs(sii[r] - bf_sii).max() < 1e-12 * scale
        assert abs(phi[r].sum() - fx[r]) < 1e-12 * max(1.0, abs(fx[r]))
        for f in range(F):
            if f not in used:
                assert phi[r, f] == 0.0 and not sii[r, f].any()


@settings(max_examples=40, deadline=None, derandomize=True, database=None)
@given(seed=st.integers(0, 10**6), F=st.integers(1, 9), depth=st.integers(0, 14), n_trees=st.integers(1, 4),
       categorical=st.booleans())
def test_library_path_tables_bit_for_bit(seed, F, depth, n_trees, categorical):
    """The library's host path preparation (no device) against the merged
    paths written out in Python from the tree arrays, on random trees."""
    import paper_2605_04497_gb300 as qts
    from test_lib_host import _expected_tables

    ens = synth.grow(seed, n_trees, depth, F, 800, 1.0, min_rows=2)
    rng = np.random.default_rng(seed)
    ens.default_left[:] = rng.integers(0, 2, ens.n_nodes).astype(np.uint8)
    if categorical:
        ens = synth.make_categorical(ens, (F - 1,), 4, seed + 3)
    got = qts.describe_paths(ens)
    rec, leaf, width = _expected_tables(ens)
    assert np.array_equal(got["path_leaf"], leaf)
    assert np.array_equal(got["path_width"], width)
    assert np.array_equal(got["records"], rec)


@settings(max_examples=40, deadline=None, derandomize=True, database=None)
@given(seed=st.integers(0, 10**6), F=st.integers(1, 9), depth=st.integers(0, 14), n_trees=st.integers(1, 4))
def test_library_alg1_program_bit_for_bit(seed, F, depth, n_trees):
    """The depth-first form's record program against the per-node data written
    out in Python from the tree arrays, on random trees."""
    import paper_2605_04497_gb300 as qts
    from test_lib_host import _expected_alg1_program

    ens = synth.grow(seed, n_trees, depth, F, 800, 1.0, min_rows=2)
    rng = np.random.default_rng(seed)
    ens.default_left[:] = rng.integers(0, 2, ens.n_nodes).astype(np.uint8)
    got = qts.describe_alg1_program(ens)
    rec, off, levels = _expected_alg1_program(ens)
    assert np.array_equal(got["tree_off"], off)
    assert np.array_equal(got["records"], rec.reshape(-1, 8))
    if len(rec):
        assert got["levels"] == levels
