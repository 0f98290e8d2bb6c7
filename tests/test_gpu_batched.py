"""The batched persistent forward + adjoint launch (graph-captured) and the
autotuner: results agree with the oracle and with the per-ensemble kernels."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import rel_err_rows

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


def hetero_batch(n, seed=4242):
    """Small heterogeneous requests: depth 2..12, F 3..40, M 1..150 (ragged)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        depth = int(rng.integers(2, 13))
        F = int(rng.integers(3, 41))
        M = int(rng.choice([1, 7, 31, 32, 33, 64, 100, 150]))
        T = int(rng.integers(1, 12))
        ens = synth.grow(seed + k, T, depth, F, 2000, 0.1, min_rows=5)
        X = synth.normal(seed + k, synth.STREAM_X, (M, F))
        G = synth.normal(seed + k, synth.STREAM_GRAD, (M, F + 1))
        out.append(synth.Workload(f"h{k}", ens, X, G))
    return out


def _prepare(q, works, grad_mask=None):
    import torch

    items, keep = [], []
    for k, w in enumerate(works):
        E = q.Ensemble.from_arrays(w.ens)
        X = torch.from_numpy(w.X).cuda()
        use_grad = grad_mask is None or grad_mask[k]
        G = torch.from_numpy(w.grad_phi).cuda() if use_grad else None
        phi = torch.empty((w.M, w.F + 1), dtype=torch.float64, device="cuda")
        dl = torch.empty(E.n_nodes, dtype=torch.float64, device="cuda") if use_grad else None
        dz = torch.empty(E.n_nodes, dtype=torch.float64, device="cuda") if use_grad else None
        items.append(dict(ens=E, X=X, grad_phi=G, phi=phi, d_leaf=dl, d_z=dz))
    return items


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_batched_matches_plain_and_oracle(qts):
    import torch

    works = hetero_batch(12)
    items = _prepare(qts, works, grad_mask=[k % 3 != 2 for k in range(len(works))])
    reqs = qts.make_requests(items)
    qts.batched_fwd_bwd(reqs)
    torch.cuda.synchronize()
    assert qts.lib().qts_batched_kernel_count() >= 2
    for w, it in zip(works, items):
        it["ens"].sync_status()
        phi = it["phi"].cpu().numpy()
        ref = oracle.shap_exact(w.ens, w.X)
        assert rel_err_rows(phi, ref).max() <= TOL32, w.name
        if it["grad_phi"] is not None:
            dl, dz = qts.shap_backward(it["ens"], it["X"], it["grad_phi"])
            assert rel(it["d_leaf"].cpu().numpy(), dl.cpu().numpy()) <= 1e-6
            assert rel(it["d_z"].cpu().numpy(), dz.cpu().numpy()) <= 1e-6
    # oracle gradient on two requests
    for k in (0, 1):
        w, it = works[k], items[k]
        dl_ref, dz_ref = oracle.grad_exact(w.ens, w.X, w.grad_phi)
        assert rel(it["d_leaf"].cpu().numpy(), dl_ref) <= TOL32
        assert rel(it["d_z"].cpu().numpy(), dz_ref) <= TOL32
    for it in items:
        it["ens"].close()


def test_graph_replay_reads_current_inputs(qts):
    import torch

    works = hetero_batch(4, seed=77)
    items = _prepare(qts, works)
    reqs = qts.make_requests(items)
    qts.batched_fwd_bwd(reqs)
    first = [it["phi"].clone() for it in items]
    qts.batched_fwd_bwd(reqs)  # replay of the cached graph
    torch.cuda.synchronize()
    for f, it in zip(first, items):  # FP32 atomics may reorder sums: compare at 1e-6 of scale
        assert rel_err_rows(it["phi"].cpu().numpy(), f.cpu().numpy()).max() <= 1e-6
    # new values in the same buffers are picked up by the replay
    items[0]["X"].mul_(-1.0)
    qts.batched_fwd_bwd(reqs)
    torch.cuda.synchronize()
    Xn = items[0]["X"].cpu().numpy()
    ref = oracle.shap_exact(works[0].ens, Xn)
    assert rel_err_rows(items[0]["phi"].cpu().numpy(), ref).max() <= TOL32
    for it in items:
        it["ens"].close()


def test_batched_rejects_duplicate_ensembles(qts):
    works = hetero_batch(2, seed=99)
    items = _prepare(qts, works)
    items[1]["ens"] = items[0]["ens"]
    with pytest.raises(qts.QtsError) as e:
        qts.batched_fwd_bwd(qts.make_requests(items))
    assert e.value.status == 1


def test_autotune_keeps_results_and_writes_cache(qts, tmp_path):
    import torch

    w = synth.workload("pairs-depth6", n_samples=300, n_trees=40, with_grad=True)
    E = qts.Ensemble.from_arrays(w.ens)
    X = torch.from_numpy(w.X).cuda()
    before = qts.shap_values(E, X).cpu().numpy()
    cache = str(tmp_path / "tune.json")
    qts.autotune(E, X, cache)
    after = qts.shap_values(E, X).cpu().numpy()
    assert rel_err_rows(after, before).max() <= 1e-6
    data = json.load(open(cache))
    assert len(data) == len(E.info()["buckets"])
    # a second ensemble of the same shape reads the cache
    E2 = qts.Ensemble.from_arrays(w.ens)
    qts.autotune(E2, X, cache)
    again = qts.shap_values(E2, X).cpu().numpy()
    assert rel_err_rows(again, before).max() <= 1e-6
    E.close()
    E2.close()


def test_batched_autotune_keeps_results(qts):
    """The batched-launch tuner changes only launch parameters: after tuning,
    phi and the gradients still match the oracle, and a later call rebuilds
    its graph with the tuned values."""
    import torch

    works = hetero_batch(6, seed=5151)
    items = _prepare(qts, works)
    reqs = qts.make_requests(items)
    chosen = qts.batched_autotune(reqs, 8, max_samples=64)
    assert chosen, "some width must carry 1% of the work"
    for D, (paths, mode, occ) in chosen.items():
        assert paths >= 32 and mode in (0, 2, 3) and occ in (0, 2, 3), (D, paths, mode, occ)
    qts.batched_fwd_bwd(reqs)
    torch.cuda.synchronize()
    for w, it in zip(works, items):
        it["ens"].sync_status()
        assert rel_err_rows(it["phi"].cpu().numpy(), oracle.shap_exact(w.ens, w.X)).max() <= TOL32, w.name
        dl_ref, dz_ref = oracle.grad_exact(w.ens, w.X, w.grad_phi)
        assert rel(it["d_leaf"].cpu().numpy(), dl_ref) <= TOL32, w.name
        assert rel(it["d_z"].cpu().numpy(), dz_ref) <= TOL32, w.name
    for it in items:
        it["ens"].close()
