"""GPU parity with categorical splits, against the FP64 oracle.

A categorical split sends x left iff x is not NaN, 0 <= x < 64 and floor(x)
is in its left set; NaN follows the default direction and every other value
goes right.  Paths merge the category sets of a feature by intersection.  The
inputs mix categories, values that are no category (negative, >= n, >= 64) and
NaN.  Tolerances as for the numerical paths: 1e-5 of max(|f(x)|, max|phi_i|)
in FP32, 1e-12 with QTS_FLAG_FP64.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import categorical_ensemble, golden_categorical_trees, rel_err_rows, sample_x

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12
CAT = (0, 2)


@pytest.fixture(scope="module")
def qts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_04497_gb300 import build as b

    b.build()
    import paper_2605_04497_gb300 as q

    return q


def case(seed, M=45, n_trees=4, depth=8, F=5):
    ens = categorical_ensemble(seed, n_trees=n_trees, depth=depth, F=F, cat_features=CAT)
    X = synth.categorical_columns(synth.normal(seed, 1, (M, F)), CAT, 6, seed)
    G = synth.normal(seed, 2, (M, F + 1))
    return ens, X, G


def cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_golden_categorical_trees(qts):
    for spec, ens in golden_categorical_trees():
        X = np.stack([sample_x(s) for s in spec["samples"]])
        want = np.array([s["phi"] for s in spec["samples"]])
        for fp64, tol in ((False, 1e-6), (True, 1e-14)):
            E = qts.Ensemble.from_arrays(ens, fp64=fp64)
            got = qts.shap_values(E, cuda(X)).cpu().numpy()
            E.sync_status()
            E.close()
            assert np.abs(got - want).max() < tol, (spec["name"], fp64)


@pytest.mark.parametrize("seed", range(4))
def test_shap_values_fp32_and_fp64(qts, seed):
    ens, X, _ = case(1800 + seed)
    ref = oracle.shap_exact(ens, X)
    for fp64, tol in ((False, TOL32), (True, TOL64)):
        E = qts.Ensemble.from_arrays(ens, fp64=fp64)
        got = qts.shap_values(E, cuda(X)).cpu().numpy()
        E.sync_status()
        E.close()
        assert rel_err_rows(got, ref).max() <= tol, fp64


def test_interactions_and_third_order(qts):
    ens, X, _ = case(1900, M=40, F=6)
    E = qts.Ensemble.from_arrays(ens)
    got2 = qts.shap_interactions(E, cuda(X)).cpu().numpy().astype(np.float64)
    got3 = qts.expand_triples(qts.shap_interactions3(E, cuda(X)).cpu().numpy().astype(np.float64), 6)
    E.sync_status()
    E.close()
    sii, phi = oracle.sii_exact(ens, X)
    scale = np.maximum(np.abs(phi.sum(1)), np.abs(phi[:, :-1]).max(1))
    err2 = np.abs(got2 - oracle.interaction_matrix(sii, phi)).reshape(len(X), -1).max(1) / scale
    err3 = np.abs(got3 - oracle.sii3_exact(ens, X)).reshape(len(X), -1).max(1) / scale
    assert err2.max() <= TOL32 and err3.max() <= TOL32


def test_backward_and_refit(qts):
    """The adjoint against the oracle's analytic gradient; a refit keeps the
    split types and category sets."""
    ens, X, G = case(2000, M=50)
    dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
    E = qts.Ensemble.from_arrays(ens)
    dl, dz = qts.shap_backward(E, cuda(X), cuda(G))
    assert rel(dl.cpu().numpy(), dl_ref) <= TOL32 and rel(dz.cpu().numpy(), dz_ref) <= TOL32
    new = ens.copy()
    new.leaf_value[:] = new.leaf_value * np.float32(-1.5)
    E.update_params(new.z, new.leaf_value)
    got = qts.shap_values(E, cuda(X)).cpu().numpy()
    E.sync_status()
    E.close()
    assert rel_err_rows(got, oracle.shap_exact(new, X)).max() <= TOL32


def test_batched_mixes_categorical_and_numerical_requests(qts):
    """One graph launch over a categorical and a numerical request: the
    categorical one takes the category-aware edge test even without NaN in its
    inputs, the numerical one keeps the fast test."""
    import torch

    ens_c, X_c, G_c = case(2100, M=300)
    X_c = np.nan_to_num(X_c, nan=70.0)  # no NaN: only the categories force the variant
    w = synth.workload("small-depth4", with_grad=True)
    items, refs = [], []
    for ens, X, G in ((ens_c, X_c, G_c), (w.ens, w.X, w.grad_phi)):
        E = qts.Ensemble.from_arrays(ens)
        items.append(dict(ens=E, X=cuda(X), grad_phi=cuda(G),
                          phi=torch.empty((X.shape[0], X.shape[1] + 1), dtype=torch.float64, device="cuda"),
                          d_leaf=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda"),
                          d_z=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda")))
        refs.append((ens, X, G))
    qts.batched_fwd_bwd(qts.make_requests(items))
    torch.cuda.synchronize()
    for it, (ens, X, G) in zip(items, refs):
        it["ens"].sync_status()
        assert rel_err_rows(it["phi"].cpu().numpy(), oracle.shap_exact(ens, X)).max() <= TOL32
        dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
        assert rel(it["d_leaf"].cpu().numpy(), dl_ref) <= TOL32
        assert rel(it["d_z"].cpu().numpy(), dz_ref) <= TOL32
        it["ens"].close()


def test_depth_first_form_rejects_categorical(qts):
    ens, X, _ = case(2200, M=8)
    E = qts.Ensemble.from_arrays(ens)
    with pytest.raises(qts.QtsError) as ei:
        qts.shap_values_alg1(E, cuda(X))
    assert ei.value.status == 4  # QTS_ERR_UNSUPPORTED
    E.close()
