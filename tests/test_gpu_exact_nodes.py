"""n_quad = EXACT_NODES (Thm 2): every bucket of paths with at most w unique
features takes ceil((w - s + 1) / 2) Gauss-Legendre points, so the results
equal the exact integrals (the oracle's Bernstein expansion) at every width,
including widths above 16 where 8 points are not exact, while narrow buckets
take fewer points than 8.  Odd point counts exercise the padded rules: node
pairs with one zero-weight node (forward, unpacked adjoint) and single nodes
(the packed fused pass)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import caterpillar_ensemble, rel_err_rows, tiny_ensemble

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-13


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


def _cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def mixed():
    """Grown trees (widths up to ~12) plus caterpillars of widths 3 to 33."""
    F = 40
    ens = synth.concat([synth.grow(8801, 6, 12, F, 3000, 0.1, min_rows=5),
                        caterpillar_ensemble(8802, [3, 9, 17, 24, 33], F)])
    X = synth.normal(8801, synth.STREAM_X, (70, F))
    G = synth.normal(8801, synth.STREAM_GRAD, (70, F + 1))
    return ens, X, G


def test_exact_forward_fp32(qts, mixed):
    ens, X, _ = mixed
    E = qts.Ensemble.from_arrays(ens)
    phi = qts.shap_values(E, _cuda(X), qts.EXACT_NODES).cpu().numpy()
    E.sync_status()
    E.close()
    assert rel_err_rows(phi, oracle.shap_exact(ens, X)).max() <= TOL32


def test_exact_forward_fp64_beyond_width_16(qts):
    """FP64 at widths 20-64: the per-bucket rule (up to 32 points) matches the
    exact expansion to rounding, where 8 points leave ~1e-12."""
    F = 80
    ens = caterpillar_ensemble(8811, [64, 48, 20], F)
    X = synth.normal(8811, synth.STREAM_X, (33, F))
    ref = oracle.shap_exact(ens, X)
    E = qts.Ensemble.from_arrays(ens, fp64=True)
    exact = qts.shap_values(E, _cuda(X), qts.EXACT_NODES).cpu().numpy()
    eight = qts.shap_values(E, _cuda(X), 8).cpu().numpy()
    E.sync_status()
    E.close()
    err_exact = rel_err_rows(exact, ref).max()
    err_eight = rel_err_rows(eight, ref).max()
    assert err_exact <= TOL64
    # the test tells the two apart: 8 points leave ~1e-12 here
    assert err_eight > 5e-13 and err_eight > 5 * err_exact, (err_eight, err_exact)


def test_exact_adjoint_fp32(qts, mixed):
    ens, X, G = mixed
    E = qts.Ensemble.from_arrays(ens)
    dl, dz = qts.shap_backward(E, _cuda(X), _cuda(G), qts.EXACT_NODES)
    E.sync_status()
    E.close()
    dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
    assert rel(dl.cpu().numpy(), dl_ref) <= TOL32
    assert rel(dz.cpu().numpy(), dz_ref) <= TOL32


def _batched(qts, cases, n_quad):
    """cases: (ens, X, G or None); one batched call; oracle checks per request."""
    import torch

    items, Es = [], []
    for ens, X, G in cases:
        E = qts.Ensemble.from_arrays(ens)
        Es.append(E)
        items.append(dict(ens=E, X=_cuda(X.astype(np.float32)), grad_phi=_cuda(G) if G is not None else None,
                          phi=torch.empty((X.shape[0], X.shape[1] + 1), dtype=torch.float64, device="cuda"),
                          d_leaf=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda") if G is not None else None,
                          d_z=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda") if G is not None else None))
    qts.batched_fwd_bwd(qts.make_requests(items), n_quad)
    torch.cuda.synchronize()
    for (ens, X, G), it, E in zip(cases, items, Es):
        E.sync_status()
        assert rel_err_rows(it["phi"].cpu().numpy(), oracle.shap_exact(ens, X)).max() <= TOL32
        if G is not None:
            dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
            assert rel(it["d_leaf"].cpu().numpy(), dl_ref) <= TOL32
            assert rel(it["d_z"].cpu().numpy(), dz_ref) <= TOL32
    for E in Es:
        E.close()


def test_exact_batched(qts, mixed):
    """Packed fused requests (widths <= 16, one node at a time), a request with
    F = 200 whose 64-sample tiles do not fit (node pairs), a forward-only
    request (node pairs below 8 points), and widths 17-33."""
    ens, X, G = mixed
    wide = synth.grow(8821, 5, 10, 200, 3000, 1.0, min_rows=2)
    Xw = synth.normal(8822, synth.STREAM_X, (33, 200))
    Gw = synth.normal(8822, synth.STREAM_GRAD, (33, 201))
    fo = tiny_ensemble(8823, n_trees=7, depth=8, F=9, n_train=3000)
    Xf = synth.normal(8823, synth.STREAM_X, (50, 9))
    _batched(qts, [(ens, X, G), (wide, Xw, Gw), (fo, Xf, None)], qts.EXACT_NODES)


def test_odd_point_count(qts):
    """n_quad = 5 on paths of at most 10 unique features (exact by Thm 2):
    forward (6 nodes, one of zero weight), adjoint, and the batched pass
    (5 single nodes packed, 6 for forward-only requests)."""
    ens = tiny_ensemble(8831, n_trees=8, depth=8, F=6, n_train=3000)
    assert oracle.path_stats(ens)[1] <= 10  # widest merged path
    X = synth.normal(8831, synth.STREAM_X, (65, 6))
    G = synth.normal(8831, synth.STREAM_GRAD, (65, 7))
    ref = oracle.shap_exact(ens, X)
    E = qts.Ensemble.from_arrays(ens)
    phi = qts.shap_values(E, _cuda(X), 5).cpu().numpy()
    dl, dz = qts.shap_backward(E, _cuda(X), _cuda(G), 5)
    E.sync_status()
    E.close()
    assert rel_err_rows(phi, ref).max() <= TOL32
    dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
    assert rel(dl.cpu().numpy(), dl_ref) <= TOL32
    assert rel(dz.cpu().numpy(), dz_ref) <= TOL32
    fo = tiny_ensemble(8832, n_trees=6, depth=7, F=6, n_train=2000)
    Xf = synth.normal(8832, synth.STREAM_X, (40, 6))
    _batched(qts, [(ens, X, G), (fo, Xf, None)], 5)
    # pairwise with 5 points (padded to 8 for widths up to 12)
    E = qts.Ensemble.from_arrays(ens)
    pairs = qts.shap_interactions(E, _cuda(X), 5).cpu().numpy().astype(np.float64)
    E.sync_status()
    E.close()
    sii, phi = oracle.sii_exact(ens, X)
    ref = oracle.interaction_matrix(sii, phi)
    scale = np.maximum(np.abs(phi.sum(1)), np.abs(phi[:, :-1]).max(1))
    assert (np.abs(pairs - ref).reshape(len(X), -1).max(1) / scale).max() <= TOL32


def test_exact_interactions_and_depth_first(qts):
    """Pairwise interactions take a rule per bucket (ceil(D / 2) points: the
    diagonal holds first-order values; padded to 4, a 4-node pass for widths up
    to 6); third order and Algorithm 1 take the rule of the ensemble's widest
    path (orders 3 and 1).  Widths up to 12, odd ones included."""
    ens = tiny_ensemble(8841, n_trees=6, depth=12, F=14, n_train=4000)
    X = synth.normal(8841, synth.STREAM_X, (35, 14))
    E = qts.Ensemble.from_arrays(ens)
    Xd = _cuda(X)
    pairs = qts.shap_interactions(E, Xd, qts.EXACT_NODES).cpu().numpy().astype(np.float64)
    sii3 = qts.expand_triples(qts.shap_interactions3(E, Xd, qts.EXACT_NODES).cpu().numpy().astype(np.float64), 14)
    alg1 = qts.shap_values_alg1(E, Xd, qts.EXACT_NODES).cpu().numpy()
    E.sync_status()
    E.close()
    sii, phi = oracle.sii_exact(ens, X)
    ref = oracle.interaction_matrix(sii, phi)
    scale = np.maximum(np.abs(phi.sum(1)), np.abs(phi[:, :-1]).max(1))
    assert (np.abs(pairs - ref).reshape(len(X), -1).max(1) / scale).max() <= TOL32
    ref3 = oracle.sii3_exact(ens, X)
    assert (np.abs(sii3 - ref3).reshape(len(X), -1).max(1) / scale).max() <= TOL32
    assert rel_err_rows(alg1, phi).max() <= TOL32
