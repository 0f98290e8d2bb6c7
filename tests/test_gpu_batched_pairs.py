"""The batched pass evaluates each pair of sibling leaves of a numerical split as
one path: the pair's leaf polynomial val_A a_A(p) + val_B a_B(p) is linear in p,
so it becomes one element (z = val_A z_A + val_B z_B, d = val_k - z for the
leaf k a sample reaches, -z for neither) of the path the two leaves share.
These cases stress that element against the FP64 oracle: pairs without shared
elements (stumps), pairs whose feature was split on above (the element's
interval comes from those splits), missing values with either default
direction, categorical parents (not merged) next to numerical ones, and every
variant of the pass: forward only, one sample per lane (wide F), two samples
per lane."""
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


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _run(qts, cases):
    """cases: (name, ens, X, G or None); one batched call; oracle checks."""
    import torch

    items, Es = [], []
    for name, ens, X, G in cases:
        E = qts.Ensemble.from_arrays(ens)
        Es.append(E)
        items.append(dict(ens=E, X=torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda(),
                          grad_phi=torch.from_numpy(G).cuda() if G is not None else None,
                          phi=torch.empty((X.shape[0], X.shape[1] + 1), dtype=torch.float64, device="cuda"),
                          d_leaf=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda") if G is not None else None,
                          d_z=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda") if G is not None else None))
    pair_paths = [E.batch_info()["n_pair_paths"] for E in Es]
    qts.batched_fwd_bwd(qts.make_requests(items))
    torch.cuda.synchronize()
    for (name, ens, X, G), it, E in zip(cases, items, Es):
        E.sync_status()
        assert rel_err_rows(it["phi"].cpu().numpy(), oracle.shap_exact(ens, X)).max() <= TOL32, name
        if G is not None:
            dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
            assert rel(it["d_leaf"].cpu().numpy(), dl_ref) <= TOL32, name
            assert rel(it["d_z"].cpu().numpy(), dz_ref) <= TOL32, name
    for E in Es:
        E.close()
    return pair_paths


def _xg(seed, M, F, nan_every=0):
    X = synth.normal(seed, synth.STREAM_X, (M, F))
    if nan_every:
        X[::nan_every, :: 3] = np.nan
    return X, synth.normal(seed, synth.STREAM_GRAD, (M, F + 1))


def test_stumps_and_repeated_features(qts):
    stumps = tiny_ensemble(9001, n_trees=9, depth=1, F=4, n_train=500)      # pairs with no other element
    rep = tiny_ensemble(9002, n_trees=8, depth=10, F=4, n_train=4000)       # pair features split on above
    mixed = tiny_ensemble(9003, n_trees=6, depth=7, F=12, n_train=3000)
    cases = []
    for k, (name, ens) in enumerate((("stumps", stumps), ("repeated", rep), ("mixed", mixed))):
        X, G = _xg(9100 + k, 70, ens.n_features)
        cases.append((name, ens, X, G))
    pairs = _run(qts, cases)
    assert all(n > 0 for n in pairs), pairs


def test_missing_values_both_default_directions(qts):
    ens = tiny_ensemble(9011, n_trees=8, depth=8, F=6, n_train=3000)
    flipped = ens.copy()
    flipped.default_left = 1 - flipped.default_left
    cases = []
    for k, (name, e) in enumerate((("nan", ens), ("nan_flipped", flipped))):
        X, G = _xg(9200 + k, 65, 6, nan_every=2)
        cases.append((name, e, X, G))
    _run(qts, cases)


def test_categorical_parents_stay_unmerged(qts):
    ens = categorical_ensemble(9021, n_trees=6, depth=7, F=5, cat_features=(0, 2))
    X, G = _xg(9300, 40, 5)
    X = synth.categorical_columns(X, (0, 2), 6, 9301)
    _run(qts, [("categorical", ens, X, G)])


def test_every_variant_of_the_pass(qts):
    """forward only; one sample per lane (F = 200, shared tile); one per lane
    with private tiles (F = 60, width above the packed cut); two per lane."""
    base = tiny_ensemble(9031, n_trees=6, depth=9, F=20, n_train=3000)
    wide = synth.grow(9032, 5, 10, 200, 3000, 1.0, min_rows=2)
    mid = synth.grow(9033, 5, 10, 60, 3000, 1.0, min_rows=2)
    X0, _ = _xg(9400, 50, 20)
    X1, G1 = _xg(9401, 33, 200)
    X2, G2 = _xg(9402, 33, 60)
    X3, G3 = _xg(9403, 129, 20)
    _run(qts, [("forward_only", base, X0, None), ("one_per_lane_shared", wide, X1, G1),
               ("one_per_lane_private", mid, X2, G2), ("two_per_lane", base.copy(), X3, G3)])
