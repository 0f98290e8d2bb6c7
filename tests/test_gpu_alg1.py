"""GPU parity of the depth-first form (qts_shap_values_alg1, Algorithm 1)
against the FP64 oracle.

Same tolerance as the path form: per sample,
    max_i |phi_gpu - phi_oracle| / max(|f(x)|, max_i |phi_oracle_i|) <= 1e-5.
The cases cover what the traversal has that the path form does not: repeated
features telescoped along the path (including an ancestor whose edge test
already failed), leaf children on either side, single-leaf trees, node groups
beyond 8 quadrature points, and missing values.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import golden_trees, rel_err_rows, sample_x, tiny_ensemble

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


def run_alg1(q, ens, X, n_quad=8):
    import torch

    E = q.Ensemble.from_arrays(ens)
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    phi = q.shap_values_alg1(E, Xd, n_quad)
    E.sync_status()
    out = phi.cpu().numpy()
    E.close()
    return out


def test_golden_trees(qts):
    """Hand-derived values, including a repeated feature and all-NaN samples."""
    for spec, ens in golden_trees():
        X = np.stack([sample_x(s) for s in spec["samples"]])
        got = run_alg1(qts, ens, X)
        want = np.array([s["phi"] for s in spec["samples"]])
        assert np.abs(got - want).max() < 1e-6, spec["name"]


def test_small_depth4_full(qts):
    w = synth.workload("small-depth4")  # M = 100: three full tiles and a ragged one
    got = run_alg1(qts, w.ens, w.X)
    ref = oracle.shap_exact(w.ens, w.X)
    assert rel_err_rows(got, ref).max() <= TOL32


@pytest.mark.parametrize("seed", range(6))
def test_repeated_features_deep(qts, seed):
    """depth 11 over 4 features: most edges repeat an ancestor's feature, often
    one whose own edge test already failed (merged o = 0)."""
    ens = tiny_ensemble(300 + seed, n_trees=4, depth=11, F=4, n_train=3000)
    X = synth.normal(300 + seed, 1, (45, 4))
    got = run_alg1(qts, ens, X)
    ref = oracle.shap_exact(ens, X)
    assert rel_err_rows(got, ref).max() <= TOL32


@pytest.mark.parametrize("n_quad", [1, 3, 8, 12, 32])
def test_node_counts_match_oracle_quadrature(qts, n_quad):
    """Any n: the same n-point rule as the oracle's quadrature (8-node groups
    padded with zero weights; 12 and 32 take several groups)."""
    ens = tiny_ensemble(410 + n_quad, n_trees=5, depth=9, F=7, n_train=2000)
    X = synth.normal(410 + n_quad, 1, (33, 7))
    got = run_alg1(qts, ens, X, n_quad)
    ref = oracle.shap_quad(ens, X, n_quad)
    assert rel_err_rows(got, ref).max() <= TOL32


def test_missing_values_and_default_directions(qts):
    """About half of the inputs are NaN; every split routes NaN by its own
    default direction."""
    ens = tiny_ensemble(520, n_trees=6, depth=8, F=6, n_train=2000)
    rng = np.random.default_rng(520)
    ens.default_left[:] = rng.integers(0, 2, ens.n_nodes).astype(np.uint8)
    X = synth.normal(520, 1, (70, 6))
    X[rng.random(X.shape) < 0.5] = np.nan
    got = run_alg1(qts, ens, X)
    ref = oracle.shap_exact(ens, X)
    assert rel_err_rows(got, ref).max() <= TOL32


def test_single_leaf_trees_and_ragged_sizes(qts):
    """Trees that are a single leaf add only to E[f]; M = 1, 31, 33 and 0."""
    import torch

    base = tiny_ensemble(610, n_trees=3, depth=6, F=5)
    stump = synth.Ensemble([0, 1], [-1], [-1], [0], [0.0], [1], [1.0], [2.5], [1], 5)
    ens = synth.concat([base, stump, base.tree(1)])
    for M in (1, 31, 33):
        X = synth.normal(611, M, (M, 5))
        got = run_alg1(qts, ens, X)
        ref = oracle.shap_exact(ens, X)
        assert rel_err_rows(got, ref).max() <= TOL32, M
    E = qts.Ensemble.from_arrays(ens)
    out = qts.shap_values_alg1(E, torch.empty((0, 5), dtype=torch.float32, device="cuda"))
    assert out.shape == (0, 6)
    E.close()


def test_agrees_with_path_form_on_xgb_shaped_ensemble(qts):
    """The 1,000-tree depth-8 ensemble at full size (M = 10,000) in the launch
    configuration the profile uses: sampled rows against the oracle, and every
    row against the path-form kernel."""
    import torch

    w = synth.workload("xgb-depth8")
    E = qts.Ensemble.from_arrays(w.ens)
    Xd = torch.from_numpy(w.X).cuda()
    a = qts.shap_values_alg1(E, Xd).cpu().numpy()
    b = qts.shap_values(E, Xd).cpu().numpy()
    E.sync_status()
    E.close()
    rows = np.array([0, 1, 31, 32, 4999, 9998, 9999])
    ref = oracle.shap_exact(w.ens, w.X[rows])
    assert rel_err_rows(a[rows], ref).max() <= TOL32
    assert rel_err_rows(a, b).max() <= 2 * TOL32


def test_deep_unbalanced_trees(qts):
    """Depth-20 unbalanced trees over F = 24 (repeated features on most deep
    paths), sampled rows against the exact expansion."""
    import torch

    w = synth.workload("deep-depth20", n_samples=512, n_trees=10)
    E = qts.Ensemble.from_arrays(w.ens)
    got = qts.shap_values_alg1(E, torch.from_numpy(w.X).cuda()).cpu().numpy()
    E.sync_status()
    E.close()
    rows = np.arange(0, 512, 37)
    ref = oracle.shap_exact(w.ens, w.X[rows])
    assert rel_err_rows(got[rows], ref).max() <= TOL32


def test_refit_rebuilds_the_traversal(qts):
    """qts_update_params drops the traversal program; the next call uses the new
    edge weights and leaf values."""
    import torch

    ens = tiny_ensemble(710, n_trees=4, depth=7, F=5)
    X = synth.normal(710, 1, (40, 5))
    E = qts.Ensemble.from_arrays(ens)
    Xd = torch.from_numpy(X).cuda()
    qts.shap_values_alg1(E, Xd)
    new = ens.copy()
    new.leaf_value[:] = new.leaf_value * 2.0 - 0.25
    new.z[:] = new.z * np.float32(0.9)  # any positive weights are accepted
    E.update_params(new.z, new.leaf_value)
    got = qts.shap_values_alg1(E, Xd).cpu().numpy()
    E.sync_status()
    E.close()
    assert rel_err_rows(got, oracle.shap_exact(new, X)).max() <= TOL32


def test_fp64_ensemble_is_rejected(qts):
    import torch

    ens = tiny_ensemble(720)
    E = qts.Ensemble.from_arrays(ens, fp64=True)
    with pytest.raises(qts.QtsError) as ei:
        qts.shap_values_alg1(E, torch.zeros((4, ens.n_features), device="cuda"))
    assert ei.value.status == 4  # QTS_ERR_UNSUPPORTED
    E.close()
