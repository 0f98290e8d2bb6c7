"""GPU parity of third-order Shapley interaction indices (qts_shap_interactions3)
against the FP64 oracle (exact Bernstein integration of Thm 1 with |S| = 3).
Per sample: max_ijk |gpu - oracle| / max(|f(x)|, max_i |phi_i|) <= 1e-5."""
import numpy as np
import pytest

import oracle
import synth
from helpers import golden_trees, sample_x, tiny_ensemble

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


def gpu3(q, ens, X, n_quad=8):
    import torch

    E = q.Ensemble.from_arrays(ens)
    out = q.shap_interactions3(E, torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda(), n_quad)
    E.sync_status()
    r = q.expand_triples(out.cpu().numpy().astype(np.float64), X.shape[1])
    E.close()
    return r


def check(got, ens, X):
    ref = oracle.sii3_exact(ens, X)
    phi = oracle.shap_exact(ens, X)
    scale = np.maximum(np.abs(phi.sum(1)), np.abs(phi[:, :-1]).max(1))
    err = np.abs(got - ref).reshape(len(X), -1).max(1) / scale
    assert err.max() <= TOL32, err.max()


def test_golden_chain_tree(qts):
    spec, ens = [g for g in golden_trees() if g[0]["name"] == "three_feature_chain"][0]
    X = np.stack([sample_x(s) for s in spec["samples"]])
    got = gpu3(qts, ens, X)
    assert abs(got[0, 0, 1, 2] - spec["samples"][0]["sii012"]) < 1e-6


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_repeated_features(qts, seed):
    ens = tiny_ensemble(1800 + seed, n_trees=10, depth=9, F=8, n_train=3000)
    X = synth.normal(1800 + seed, 1, (45, 8))
    check(gpu3(qts, ens, X), ens, X)


def test_missing_values_and_ragged(qts):
    ens = tiny_ensemble(1900, n_trees=6, depth=7, F=7, n_train=2000)
    X = synth.normal(1900, 1, (33, 7))
    X[::4, 2] = np.nan
    X[3, :] = np.nan
    check(gpu3(qts, ens, X), ens, X)
    check(gpu3(qts, ens, X[:1]), ens, X[:1])


def test_interaction_sized_config(qts):
    """The 500-tree depth-6 F = 30 shape (subset of trees and samples)."""
    w = synth.workload("pairs-depth6", n_samples=40, n_trees=25)
    check(gpu3(qts, w.ens, w.X), w.ens, w.X)


def test_rejects_too_many_features(qts):
    import torch

    ens = tiny_ensemble(1950, n_trees=2, depth=4, F=200, n_train=500)
    E = qts.Ensemble.from_arrays(ens)
    with pytest.raises(qts.QtsError) as e:
        qts.shap_interactions3(E, torch.zeros((4, 200), device="cuda"))
    assert e.value.status == 4
    E.close()
