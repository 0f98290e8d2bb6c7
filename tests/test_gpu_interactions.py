"""GPU parity of pairwise interactions (qts_shap_interactions) against the
FP64 oracle (exact Bernstein integration of Thm 1 with |S| = 2).

Per sample, max over the (F+1)^2 matrix of |gpu - oracle| divided by
max(|f(x)|, max_i |phi_i|) must be <= 1e-5 (FP32 output, FP64 accumulation).
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from helpers import tiny_ensemble

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def qts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_04497_gb300 import build as b

    b.build()
    import paper_2605_04497_gb300 as q

    return q


def gpu_int(q, ens, X, n_quad=8):
    import torch

    E = q.Ensemble.from_arrays(ens)
    out = q.shap_interactions(E, torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda(), n_quad)
    E.sync_status()
    r = out.cpu().numpy().astype(np.float64)
    E.close()
    return r


def check(got, ens, X):
    sii, phi = oracle.sii_exact(ens, X)
    ref = oracle.interaction_matrix(sii, phi)
    scale = np.maximum(np.abs(phi.sum(1)), np.abs(phi[:, :-1]).max(1))
    err = np.abs(got - ref).reshape(len(X), -1).max(1) / scale
    assert err.max() <= TOL32, err.max()
    # structure: symmetric, rows sum to phi_i, bias at [F, F]
    F = X.shape[1]
    assert np.abs(got - np.transpose(got, (0, 2, 1))).max() <= 1e-6 * scale.max()
    rows = got[:, :F, :F].sum(axis=2)
    assert (np.abs(rows - phi[:, :F]).max(1) / scale).max() <= TOL32
    assert np.all(got[:, :F, F] == 0) and np.all(got[:, F, :F] == 0)


def test_pairs_depth6_small(qts):
    w = synth.workload("pairs-depth6", n_samples=70, n_trees=25)
    check(gpu_int(qts, w.ens, w.X), w.ens, w.X)


def test_repeated_features_and_missing(qts):
    ens = tiny_ensemble(1101, n_trees=12, depth=9, F=6, n_train=3000)
    X = synth.normal(1101, 1, (45, 6))
    X[::5, 3] = np.nan
    check(gpu_int(qts, ens, X), ens, X)


def test_many_features_global_accumulator(qts):
    """F = 80: the pair tile no longer fits shared memory; sums go straight to
    the FP64 accumulator."""
    ens = tiny_ensemble(1201, n_trees=6, depth=7, F=80, n_train=3000)
    X = synth.normal(1201, 1, (40, 80))
    check(gpu_int(qts, ens, X), ens, X)


def test_whole_matrix_sums_to_prediction(qts):
    ens = tiny_ensemble(1301, n_trees=8, depth=6, F=10, n_train=2000)
    X = synth.normal(1301, 1, (33, 10))
    got = gpu_int(qts, ens, X)
    f = oracle.predict(ens, X)
    assert np.abs(got.sum(axis=(1, 2)) - f).max() <= TOL32 * max(1.0, np.abs(f).max())


def test_pairs_depth6_full_size_sampled_rows(qts):
    """The 500-tree depth-6 interaction workload at full size (F = 30, M = 2,000)."""
    w = synth.workload("pairs-depth6")
    got = gpu_int(qts, w.ens, w.X)
    rows = np.r_[0:6, 1000:1004, 1994:2000]
    check(got[rows], w.ens, w.X[rows])


def test_sibling_pair_paths(qts):
    """The call runs on the tables where each pair of sibling leaves of a
    numerical split is one path whose last element (out of feature order, after
    the padding) stands for both leaves: stumps (paths with only that element),
    the split feature repeated above, missing values with either default
    direction, and the any-order kernel (per-leaf tables) as a second
    reference."""
    import torch

    stumps = tiny_ensemble(1401, n_trees=9, depth=1, F=4, n_train=500)
    X = synth.normal(1401, 1, (37, 4))
    check(gpu_int(qts, stumps, X), stumps, X)
    rep = tiny_ensemble(1402, n_trees=8, depth=10, F=4, n_train=4000)
    X = synth.normal(1402, 1, (41, 4))
    X[::3, 1] = np.nan
    check(gpu_int(qts, rep, X), rep, X)
    flipped = rep.copy()
    flipped.default_left = 1 - flipped.default_left
    check(gpu_int(qts, flipped, X), flipped, X)
    E = qts.Ensemble.from_arrays(rep)
    assert E.batch_info()["n_pair_paths"] > 0
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    pairs = qts.shap_interactions(E, Xd).cpu().numpy().astype(np.float64)
    leaves = qts.shap_interactions_order(E, Xd, 2).cpu().numpy().astype(np.float64)
    E.sync_status()
    E.close()
    sii = np.stack([2.0 * pairs[:, a, b] for a, b in itertools.combinations(range(4), 2)], axis=1)
    scale = np.abs(pairs).reshape(len(X), -1).max(1)[:, None]
    assert (np.abs(sii - leaves) / scale).max() <= 2 * TOL32
