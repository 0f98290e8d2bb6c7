"""Fashion-MNIST-shaped inputs (F = 784 features, deep trees whose merged paths
reach 40-52 unique features; the paper's Table 1 FMNIST models): forward,
adjoint and the batched fused pass against the FP64 oracle.

At this width the per-block sample and accumulator tiles take most of the
227 KB of shared memory; the kernels stage fewer path records at a time, and
the FP64 forward adds straight into phi instead of a shared FP64 tile."""
import numpy as np
import pytest

import oracle
import synth
from helpers import caterpillar_ensemble, rel_err_rows

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12
F = 784


@pytest.fixture(scope="module")
def qts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_04497_gb300 import build as b

    b.build()
    import paper_2605_04497_gb300 as q

    return q


@pytest.fixture(scope="module")
def wide():
    # grown trees (paths up to ~25 unique features) plus caterpillars whose
    # longest paths have 33-48 unique features (widths 40 and 48)
    ens = synth.concat([synth.grow(7840, 6, 52, F, 3000, 0.1, min_rows=5),
                        caterpillar_ensemble(7842, [48, 44, 40, 33], F)])
    X = synth.normal(7840, synth.STREAM_X, (40, F))  # one full sample tile and a ragged one
    G = synth.normal(7840, synth.STREAM_GRAD, (40, F + 1))
    return ens, X, G


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_wide_paths_reach_the_wide_buckets(qts, wide):
    ens, X, G = wide
    info = qts.describe(ens)
    assert info["max_unique"] == 48, info["max_unique"]
    assert {40, 48} <= {w for w, n in info["buckets"] if n > 0}


def test_forward_fp32_f784(qts, wide):
    import torch

    ens, X, G = wide
    E = qts.Ensemble.from_arrays(ens)
    phi = qts.shap_values(E, torch.from_numpy(X).cuda()).cpu().numpy()
    E.sync_status()
    E.close()
    assert rel_err_rows(phi, oracle.shap_exact(ens, X)).max() <= TOL32


def test_forward_fp64_f784(qts, wide):
    """FP64 mode against the oracle's own 8-point quadrature (paths beyond 16
    unique features are integrated inexactly by 8 points, Thm 2, on both sides)."""
    import torch

    ens, X, G = wide
    E = qts.Ensemble.from_arrays(ens, fp64=True)
    phi = qts.shap_values(E, torch.from_numpy(X).cuda()).cpu().numpy()
    E.sync_status()
    E.close()
    ref = oracle.shap_quad(ens, X, 8)
    scale = np.maximum(np.abs(ref.sum(1)), np.abs(ref[:, :-1]).max(1))
    assert (np.abs(phi - ref).max(1) / scale).max() <= TOL64


def test_adjoint_f784(qts, wide):
    import torch

    ens, X, G = wide
    E = qts.Ensemble.from_arrays(ens)
    dl, dz = qts.shap_backward(E, torch.from_numpy(X).cuda(), torch.from_numpy(G).cuda())
    E.sync_status()
    E.close()
    dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
    assert rel(dl.cpu().numpy(), dl_ref) <= TOL32
    assert rel(dz.cpu().numpy(), dz_ref) <= TOL32


def test_batched_f784(qts, wide):
    import torch

    ens, X, G = wide
    E = qts.Ensemble.from_arrays(ens)
    it = dict(ens=E, X=torch.from_numpy(X).cuda(), grad_phi=torch.from_numpy(G).cuda(),
              phi=torch.empty((X.shape[0], F + 1), dtype=torch.float64, device="cuda"),
              d_leaf=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda"),
              d_z=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda"))
    qts.batched_fwd_bwd(qts.make_requests([it]))
    torch.cuda.synchronize()
    E.sync_status()
    assert rel_err_rows(it["phi"].cpu().numpy(), oracle.shap_exact(ens, X)).max() <= TOL32
    dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
    assert rel(it["d_leaf"].cpu().numpy(), dl_ref) <= TOL32
    assert rel(it["d_z"].cpu().numpy(), dz_ref) <= TOL32
    E.close()


def test_loader_refuses_above_the_limit(qts):
    ens = synth.grow(7841, 1, 4, 900, 200, 0.1, min_rows=5)
    with pytest.raises(qts.QtsError) as e:
        qts.Ensemble.from_arrays(ens)
    assert e.value.status == 4  # QTS_ERR_UNSUPPORTED
