"""GPU parity of Shapley interactions of any order (qts_shap_interactions_order)
against the FP64 oracle's exact order-s expansion.

Per sample, max over subsets |SII_gpu - SII_oracle| / max(|f(x)|, max_i |phi_i|)
<= 1e-5 (FP32).  Orders 2 and 3 are also checked against the dedicated pair and
triple kernels, which pins the compact layout from the GPU side.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from helpers import categorical_ensemble, tiny_ensemble

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


def scale_of(ens, X):
    phi = oracle.shap_exact(ens, X)
    return np.maximum(np.abs(phi.sum(1)), np.abs(phi[:, :-1]).max(1))


@pytest.mark.parametrize("order", [7, 8])
def test_orders_7_and_8_against_exact_expansion(qts, order):
    """The two highest orders the entry point accepts: depth 10 over F = 9, so
    paths reach 8 unique features and order 8 is not identically zero."""
    ens = tiny_ensemble(2707, n_trees=4, depth=10, F=9, n_train=3000)
    X = synth.normal(2707, 1, (45, 9))
    E = qts.Ensemble.from_arrays(ens)
    assert E.info()["max_unique"] >= order
    got = qts.shap_interactions_order(E, cuda(X), order).cpu().numpy().astype(np.float64)
    E.sync_status()
    E.close()
    ref = oracle.sii_order_exact(ens, X, order)
    assert np.abs(ref).max() > 0
    err = np.abs(got - ref).max(axis=1) / scale_of(ens, X)
    assert err.max() <= TOL32, (order, err.max())


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6])
def test_against_exact_expansion(qts, order):
    """depth 9 over F = 8 (repeated features, paths up to 8 unique features),
    M = 45: two sample tiles, one ragged."""
    ens = tiny_ensemble(2600 + order, n_trees=4, depth=9, F=8, n_train=3000)
    X = synth.normal(2600 + order, 1, (45, 8))
    E = qts.Ensemble.from_arrays(ens)
    got = qts.shap_interactions_order(E, cuda(X), order).cpu().numpy().astype(np.float64)
    E.sync_status()
    E.close()
    ref = oracle.sii_order_exact(ens, X, order)
    err = np.abs(got - ref).max(axis=1) / scale_of(ens, X)
    assert err.max() <= TOL32, (order, err.max())


def test_orders_two_and_three_match_the_dedicated_kernels(qts):
    ens = tiny_ensemble(2700, n_trees=5, depth=8, F=7, n_train=2000)
    X = synth.normal(2700, 1, (40, 7))
    E = qts.Ensemble.from_arrays(ens)
    o2 = qts.shap_interactions_order(E, cuda(X), 2).cpu().numpy().astype(np.float64)
    o3 = qts.shap_interactions_order(E, cuda(X), 3).cpu().numpy().astype(np.float64)
    pair = qts.shap_interactions(E, cuda(X)).cpu().numpy().astype(np.float64)
    tri = qts.shap_interactions3(E, cuda(X)).cpu().numpy().astype(np.float64)
    E.sync_status()
    E.close()
    pairs = list(itertools.combinations(range(7), 2))
    from_pair = np.stack([2.0 * pair[:, a, b] for a, b in pairs], axis=1)  # off-diagonal holds SII/2
    sc = scale_of(ens, X)[:, None]
    assert (np.abs(o2 - from_pair) / sc).max() <= 2 * TOL32
    assert (np.abs(o3 - tri) / sc).max() <= 2 * TOL32


def test_wide_paths(qts):
    """Order 4 on paths of up to 16 unique features (one depth-16 tree over
    F = 16): 8 points are exact for d <= 2*8 + 4 - 1 (Thm 2), so the GPU
    matches the exact expansion."""
    ens = tiny_ensemble(2650, n_trees=1, depth=16, F=16, n_train=400)
    _, dmax, _ = oracle.path_stats(ens)
    assert dmax >= 12
    X = synth.normal(2650, 1, (12, 16))
    E = qts.Ensemble.from_arrays(ens)
    got = qts.shap_interactions_order(E, cuda(X), 4).cpu().numpy().astype(np.float64)
    E.sync_status()
    E.close()
    ref = oracle.sii_order_exact(ens, X, 4)
    assert (np.abs(got - ref).max(axis=1) / scale_of(ens, X)).max() <= TOL32


def test_categorical_and_missing_values(qts):
    ens = categorical_ensemble(2800, n_trees=3, depth=8, F=6, cat_features=(1, 3))
    X = synth.categorical_columns(synth.normal(2800, 1, (37, 6)), (1, 3), 6, 2800)
    E = qts.Ensemble.from_arrays(ens)
    got = qts.shap_interactions_order(E, cuda(X), 4).cpu().numpy().astype(np.float64)
    E.sync_status()
    E.close()
    ref = oracle.sii_order_exact(ens, X, 4)
    assert (np.abs(got - ref).max(axis=1) / scale_of(ens, X)).max() <= TOL32


def test_argument_errors(qts):
    import torch

    ens = tiny_ensemble(2900, F=5)
    E = qts.Ensemble.from_arrays(ens)
    for bad in (1, 9):
        with pytest.raises(qts.QtsError) as ei:
            qts.shap_interactions_order(E, torch.zeros((4, 5), device="cuda"), bad,
                                        out=torch.empty((4, 1), device="cuda"))
        assert ei.value.status == 1
    out = qts.shap_interactions_order(E, torch.zeros((0, 5), device="cuda"), 4)
    assert out.shape == (0, 5)
    E.close()
