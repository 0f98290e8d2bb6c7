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
