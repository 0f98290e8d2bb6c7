"""GPU parity at the library's stated limits: merged paths of up to 62 unique
features (the 40-64 buckets and the batched kernel's widest register classes)
and F = 640 features (QTS_MAX_FEATURES)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import caterpillar_ensemble, rel_err_rows, tiny_ensemble

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12
WIDE = (25, 36, 45, 52, 62)  # buckets 28, 40, 48, 56, 64


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


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def wide_case(M=40):
    ens = caterpillar_ensemble(3100, WIDE, 64)
    X = synth.normal(3100, 1, (M, 64))
    G = synth.normal(3100, 2, (M, 65))
    return ens, X, G


def test_widest_paths_forward(qts):
    """32 points are exact for d <= 64 (Thm 2): FP32 within its tolerance and
    FP64 to 1e-12 of the exact expansion."""
    ens, X, _ = wide_case()
    _, dmax, _ = oracle.path_stats(ens)
    assert dmax == 62
    ref = oracle.shap_exact(ens, X)
    for fp64, tol in ((False, TOL32), (True, TOL64)):
        E = qts.Ensemble.from_arrays(ens, fp64=fp64)
        got = qts.shap_values(E, cuda(X), 32).cpu().numpy()
        E.sync_status()
        E.close()
        assert rel_err_rows(got, ref).max() <= tol, fp64


def test_widest_paths_backward_and_batched(qts):
    import torch

    ens, X, G = wide_case()
    dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
    E = qts.Ensemble.from_arrays(ens)
    dl, dz = qts.shap_backward(E, cuda(X), cuda(G), 32)
    assert rel(dl.cpu().numpy(), dl_ref) <= TOL32 and rel(dz.cpu().numpy(), dz_ref) <= TOL32
    # batched fused pass: the 32- and 64-wide register classes
    phi = torch.empty((X.shape[0], 65), dtype=torch.float64, device="cuda")
    bl = torch.empty(E.n_nodes, dtype=torch.float64, device="cuda")
    bz = torch.empty(E.n_nodes, dtype=torch.float64, device="cuda")
    qts.batched_fwd_bwd(qts.make_requests([dict(ens=E, X=cuda(X), grad_phi=cuda(G), phi=phi, d_leaf=bl, d_z=bz)]),
                        32)
    torch.cuda.synchronize()
    E.sync_status()
    assert rel_err_rows(phi.cpu().numpy(), oracle.shap_exact(ens, X)).max() <= TOL32
    assert rel(bl.cpu().numpy(), dl_ref) <= TOL32 and rel(bz.cpu().numpy(), dz_ref) <= TOL32
    E.close()


def test_max_features(qts):
    """F = 640: the sample tiles and phi tiles at their largest."""
    import torch

    ens = tiny_ensemble(3003, n_trees=3, depth=8, F=640, n_train=3000)
    X = synth.normal(3003, 1, (40, 640))
    G = synth.normal(3003, 2, (40, 641))
    ref = oracle.shap_exact(ens, X)
    dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
    E = qts.Ensemble.from_arrays(ens)
    got = qts.shap_values(E, cuda(X)).cpu().numpy()
    assert rel_err_rows(got, ref).max() <= TOL32
    dl, dz = qts.shap_backward(E, cuda(X), cuda(G))
    assert rel(dl.cpu().numpy(), dl_ref) <= TOL32 and rel(dz.cpu().numpy(), dz_ref) <= TOL32
    w = synth.workload("small-depth4", with_grad=True)
    E2 = qts.Ensemble.from_arrays(w.ens)
    items = []
    for e, x, g in ((E, X, G), (E2, w.X, w.grad_phi)):
        items.append(dict(ens=e, X=cuda(x), grad_phi=cuda(g),
                          phi=torch.empty((x.shape[0], x.shape[1] + 1), dtype=torch.float64, device="cuda"),
                          d_leaf=torch.empty(e.n_nodes, dtype=torch.float64, device="cuda"),
                          d_z=torch.empty(e.n_nodes, dtype=torch.float64, device="cuda")))
    qts.batched_fwd_bwd(qts.make_requests(items))
    torch.cuda.synchronize()
    E.sync_status()
    assert rel_err_rows(items[0]["phi"].cpu().numpy(), ref).max() <= TOL32
    assert rel(items[0]["d_leaf"].cpu().numpy(), dl_ref) <= TOL32
    assert rel(items[0]["d_z"].cpu().numpy(), dz_ref) <= TOL32
    assert rel_err_rows(items[1]["phi"].cpu().numpy(), oracle.shap_exact(w.ens, w.X)).max() <= TOL32
    E.close()
    E2.close()
