"""GPU parity of the adjoint (qts_shap_backward) and the autograd wrapper.

L = sum_s sum_f grad_phi[s,f] phi[s,f].  Tolerances: FP32 kernels
max|d - d_oracle| <= 1e-5 * max|d_oracle| per gradient array; FP64 mode 1e-12.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import golden_trees, sample_x, tiny_ensemble

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


@pytest.fixture(scope="module")
def qts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_04497_gb300 import build as b

    b.build()
    import paper_2605_04497_gb300 as q

    return q


def gpu_grad(q, ens, X, G, n_quad=8, fp64=False):
    import torch

    E = q.Ensemble.from_arrays(ens, fp64=fp64)
    dl, dz = q.shap_backward(E, torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda(),
                             torch.from_numpy(np.ascontiguousarray(G, np.float32)).cuda(), n_quad)
    E.sync_status()
    out = dl.cpu().numpy(), dz.cpu().numpy()
    E.close()
    return out


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_small_depth4_gradients(qts):
    w = synth.workload("small-depth4", with_grad=True)
    dl_ref, dz_ref = oracle.grad_exact(w.ens, w.X, w.grad_phi)
    dl, dz = gpu_grad(qts, w.ens, w.X, w.grad_phi)
    assert rel(dl, dl_ref) <= TOL32 and rel(dz, dz_ref) <= TOL32
    roots = w.ens.node_offsets[:-1]
    assert np.all(dz[roots] == 0) and np.all(dl[w.ens.left >= 0] == 0)
    dl64, dz64 = gpu_grad(qts, w.ens, w.X, w.grad_phi, fp64=True)
    assert rel(dl64, dl_ref) <= TOL64 and rel(dz64, dz_ref) <= TOL64


@pytest.mark.parametrize("seed", [1, 2])
def test_repeated_features_chain_rule(qts, seed):
    """Merged elements spread dL/dz over several edges (product rule)."""
    ens = tiny_ensemble(700 + seed, n_trees=10, depth=10, F=5, n_train=3000)
    X = synth.normal(700 + seed, 1, (70, 5))
    G = synth.normal(700 + seed, 2, (70, 6))
    dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
    dl, dz = gpu_grad(qts, ens, X, G)
    assert rel(dl, dl_ref) <= TOL32 and rel(dz, dz_ref) <= TOL32
    dl64, dz64 = gpu_grad(qts, ens, X, G, fp64=True)
    assert rel(dl64, dl_ref) <= TOL64 and rel(dz64, dz_ref) <= TOL64


def test_missing_values_and_single_leaf(qts):
    spec, ens = golden_trees()[0]
    stump = synth.Ensemble([0, 1], [-1], [-1], [-1], [0], [0], [1], [2.5], [1], 2)
    both = synth.concat([tiny_ensemble(801, n_trees=3, depth=5, F=2, n_train=500), ens, stump])
    X = synth.normal(801, 1, (40, 2))
    X[::4, 0] = np.nan
    X[1, :] = np.nan
    G = synth.normal(801, 2, (40, 3))
    dl_ref, dz_ref = oracle.grad_exact(both, X, G)
    dl, dz = gpu_grad(qts, both, X, G)
    assert rel(dl, dl_ref) <= TOL32 and rel(dz, dz_ref) <= TOL32
    assert abs(dl[-1] - G[:, 2].astype(np.float64).sum()) < 1e-9


def test_fp64_finite_differences_of_gpu_forward(qts):
    """phi is linear in each leaf value and in each edge weight, so a central
    difference of the GPU's FP64 forward is exact up to rounding."""
    import torch

    ens = tiny_ensemble(901, n_trees=3, depth=6, F=6, n_train=800)
    X = synth.normal(901, 1, (33, 6))
    G = synth.normal(901, 2, (33, 7))
    dl, dz = gpu_grad(qts, ens, X, G, fp64=True)
    Xd = torch.from_numpy(X).cuda()
    Gd = torch.from_numpy(G).double().cuda()

    def loss(e):
        E = qts.Ensemble.from_arrays(e, fp64=True)
        v = float((qts.shap_values(E, Xd) * Gd).sum())
        E.close()
        return v

    rng = np.random.default_rng(0)
    leaves = np.flatnonzero(ens.left < 0)
    nonroot = np.setdiff1d(np.arange(ens.n_nodes), ens.node_offsets[:-1])
    for n in rng.choice(leaves, 6, replace=False):
        ep, em = ens.copy(), ens.copy()
        ep.leaf_value[n] += np.float32(0.5)
        em.leaf_value[n] -= np.float32(0.5)
        fd = (loss(ep) - loss(em)) / (float(ep.leaf_value[n]) - float(em.leaf_value[n]))
        assert abs(fd - dl[n]) <= 1e-10 * max(1.0, abs(dl[n]))
    for n in rng.choice(nonroot, 8, replace=False):
        ep, em = ens.copy(), ens.copy()
        h = np.float32(min(0.01, 0.5 * float(ens.z[n])))
        ep.z[n] += h
        em.z[n] -= h
        fd = (loss(ep) - loss(em)) / (float(ep.z[n]) - float(em.z[n]))
        assert abs(fd - dz[n]) <= 1e-9 * max(1.0, abs(dz[n]))


def test_xgb_depth8_full_size_sampled_leaves(qts):
    """The 1,000-tree depth-8 ensemble (M = 10,000) at full size; the oracle computes the gradient of sampled
    leaves exactly (d_leaf[v] and d_z[v] only depend on v's own path)."""
    import torch

    w = synth.workload("xgb-depth8", with_grad=True)
    E = qts.Ensemble.from_arrays(w.ens)
    dl, dz = qts.shap_backward(E, torch.from_numpy(w.X).cuda(), torch.from_numpy(w.grad_phi).cuda())
    E.sync_status()
    dl, dz = dl.cpu().numpy(), dz.cpu().numpy()
    E.close()
    leaves = np.flatnonzero(w.ens.left < 0)
    pick = np.random.default_rng(1).choice(leaves, 24, replace=False)
    dl_ref, dz_ref = oracle.grad_exact(w.ens, w.X, w.grad_phi, leaves=pick)
    scale_l = np.abs(dl_ref[pick]).max()
    scale_z = np.abs(dz_ref[pick]).max()
    assert np.abs(dl[pick] - dl_ref[pick]).max() <= TOL32 * scale_l
    assert np.abs(dz[pick] - dz_ref[pick]).max() <= TOL32 * scale_z


def test_autograd_function(qts):
    import torch

    w = synth.workload("small-depth4", n_samples=40, with_grad=True)
    E = qts.Ensemble.from_arrays(w.ens)
    lv = torch.tensor(w.ens.leaf_value, requires_grad=True)
    z = torch.tensor(w.ens.z, requires_grad=True)
    X = torch.from_numpy(w.X).cuda()
    phi = qts.QTreeShapFn.apply(E, lv, z, X)
    G = torch.from_numpy(w.grad_phi).cuda()
    (phi * G.double()).sum().backward()
    dl_ref, dz_ref = oracle.grad_exact(w.ens, w.X, w.grad_phi)
    assert rel(lv.grad.numpy().astype(np.float64), dl_ref) <= 1e-5
    assert rel(z.grad.numpy().astype(np.float64), dz_ref) <= 1e-5
    # a changed parameter vector is pushed to the device tables
    lv2 = torch.tensor(w.ens.leaf_value * 2.0)
    phi2 = qts.QTreeShapFn.apply(E, lv2, z.detach(), X)
    assert torch.allclose(phi2[:, :-1], 2 * phi[:, :-1].detach(), rtol=1e-5, atol=1e-7)
    E.close()
