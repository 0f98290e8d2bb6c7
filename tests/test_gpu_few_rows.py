"""Calls with few explained rows (M <= 16, the setting of the paper's
interaction timings: 100 rows, 1 row): the kernels map lanes to (path, sample)
pairs instead of one sample per lane.  First order, pairwise (pred_interactions
layout), third order and orders 4-5 against the FP64 oracle at M = 1, 7 and 16,
with repeated features, missing values and categorical splits."""
import numpy as np
import pytest

import oracle
import synth
from helpers import categorical_ensemble, rel_err_rows, tiny_ensemble

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


def cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def scale_of(phi):
    return np.maximum(np.abs(phi.sum(1)), np.abs(phi[:, :-1]).max(1))


def _ensembles():
    deep = synth.workload("deep-depth20", n_samples=16, n_trees=6)  # widths above 16 (padded)
    xgb = synth.workload("xgb-depth8", n_samples=16, n_trees=60)
    rep = tiny_ensemble(3301, n_trees=10, depth=9, F=7, n_train=3000)  # repeated features
    X_rep = synth.normal(3301, 1, (16, 7))
    X_rep[::3, 2] = np.nan
    return [("deep20", deep.ens, deep.X), ("xgb8", xgb.ens, xgb.X), ("repeated_nan", rep, X_rep)]


@pytest.mark.parametrize("M", [1, 7, 16])
def test_first_order_few_rows(qts, M):
    for name, ens, X in _ensembles():
        E = qts.Ensemble.from_arrays(ens)
        phi = qts.shap_values(E, cuda(X[:M])).cpu().numpy()
        E.sync_status()
        E.close()
        assert rel_err_rows(phi, oracle.shap_exact(ens, X[:M])).max() <= TOL32, (name, M)


@pytest.mark.parametrize("M", [1, 7])
def test_first_order_few_rows_categorical(qts, M):
    ens = categorical_ensemble(3401, n_trees=5, depth=7, F=5)
    X = synth.categorical_columns(synth.normal(3401, 1, (M, 5)), (0, 2), 6, 3402)
    E = qts.Ensemble.from_arrays(ens)
    phi = qts.shap_values(E, cuda(X)).cpu().numpy()
    E.sync_status()
    E.close()
    assert rel_err_rows(phi, oracle.shap_exact(ens, X)).max() <= TOL32


@pytest.mark.parametrize("M", [1, 7, 16])
def test_pairwise_few_rows(qts, M):
    w = synth.workload("pairs-depth6", n_samples=16, n_trees=40)
    for name, ens, X in [("pairs6", w.ens, w.X)] + _ensembles()[2:]:
        if ens.n_features > 40:
            continue
        E = qts.Ensemble.from_arrays(ens)
        got = qts.shap_interactions(E, cuda(X[:M])).cpu().numpy().astype(np.float64)
        E.sync_status()
        E.close()
        sii, phi = oracle.sii_exact(ens, X[:M])
        ref = oracle.interaction_matrix(sii, phi)
        err = np.abs(got - ref).reshape(M, -1).max(1) / scale_of(phi)
        assert err.max() <= TOL32, (name, M, err.max())


@pytest.mark.parametrize("M", [1, 7])
def test_third_order_few_rows(qts, M):
    ens = tiny_ensemble(3501, n_trees=6, depth=9, F=8, n_train=3000)
    X = synth.normal(3501, 1, (M, 8))
    E = qts.Ensemble.from_arrays(ens)
    got = qts.expand_triples(qts.shap_interactions3(E, cuda(X)).cpu().numpy(), 8).astype(np.float64)
    E.sync_status()
    E.close()
    ref = oracle.sii3_exact(ens, X)
    err = np.abs(got - ref).reshape(M, -1).max(1) / scale_of(oracle.shap_exact(ens, X))
    assert err.max() <= TOL32, err.max()


@pytest.mark.parametrize("M,order", [(1, 4), (7, 4), (1, 5), (16, 2)])
def test_any_order_few_rows(qts, M, order):
    ens = tiny_ensemble(3600 + order, n_trees=5, depth=10, F=9, n_train=3000)
    X = synth.normal(3600 + order, 1, (M, 9))
    E = qts.Ensemble.from_arrays(ens)
    got = qts.shap_interactions_order(E, cuda(X), order).cpu().numpy().astype(np.float64)
    E.sync_status()
    E.close()
    ref = oracle.sii_order_exact(ens, X, order)
    err = np.abs(got - ref).max(axis=1) / scale_of(oracle.shap_exact(ens, X))
    assert err.max() <= TOL32, (M, order, err.max())
