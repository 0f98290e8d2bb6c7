"""The 64-ensemble batch at full size, in the launch configuration the
benchmark times (tuned on 1,024-sample prefixes, then one batched call with
8 points): phi on sampled rows and d_leaf / d_z at sampled leaves of every
request the oracle can expand in seconds (at most 1.5 million leaves), plus
one row of every larger request that carries at least 5% of the work, against
the FP64 oracle at 1e-5.  Takes about three minutes on one GB300."""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
import synth

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


def _plan(works, rows_per=2, leaves_per=16, small_leaves=1_500_000, heavy_share=0.05):
    work = np.array([w.M * w.ens.n_leaves for w in works], dtype=np.float64)
    share = work / work.sum()
    plan = {}
    for k, w in enumerate(works):
        small = w.ens.n_leaves <= small_leaves
        if w.M == 0 or (not small and share[k] < heavy_share):
            continue
        rows = np.unique(np.linspace(0, w.M - 1, min(rows_per if small else 1, w.M)).astype(int))
        leaves = np.flatnonzero(w.ens.left < 0)
        rng = np.random.default_rng(7000 + k)
        plan[k] = (rows, np.sort(rng.choice(leaves, size=min(leaves_per, len(leaves)), replace=False)))
    return plan, float(share[list(plan)].sum())


def test_batch64_full_size_against_the_oracle(qts):
    import torch

    works = synth.batch_config()
    ens = [qts.Ensemble.from_arrays(w.ens) for w in works]
    items = [dict(ens=e, X=torch.from_numpy(w.X).cuda(), grad_phi=torch.from_numpy(w.grad_phi).cuda(),
                  phi=torch.empty((w.M, w.F + 1), dtype=torch.float64, device="cuda"),
                  d_leaf=torch.empty(e.n_nodes, dtype=torch.float64, device="cuda"),
                  d_z=torch.empty(e.n_nodes, dtype=torch.float64, device="cuda")) for e, w in zip(ens, works)]
    reqs = qts.make_requests(items)
    qts.batched_autotune(reqs, 8, max_samples=1024)
    qts.batched_fwd_bwd(reqs, 8)
    torch.cuda.synchronize()
    for e in ens:
        e.sync_status()

    plan, share = _plan(works)
    assert share > 0.99, share  # the checked requests carry nearly all the work

    def phi_ref(k):
        return oracle.shap_exact(works[k].ens, works[k].X[plan[k][0]], n_threads=2)

    def grad_ref(k):
        w, pick = works[k], plan[k][1]
        dl, dz = oracle.grad_exact(w.ens, w.X, w.grad_phi, leaves=pick, n_threads=4)
        return dl[pick], dz[pick]

    with cf.ThreadPoolExecutor(max_workers=oracle.threads()) as ex:
        fut = {k: (ex.submit(phi_ref, k), ex.submit(grad_ref, k)) for k in plan}
        for k, (fp, fg) in fut.items():
            rows, pick = plan[k]
            ref = fp.result()
            got = items[k]["phi"][torch.from_numpy(rows).cuda()].cpu().numpy()
            scale = np.maximum(np.abs(ref.sum(1)), np.abs(ref[:, :-1]).max(1))
            assert (np.abs(got - ref).max(1) / np.maximum(scale, 1e-300)).max() <= TOL32, k
            rl, rz = fg.result()
            idx = torch.from_numpy(pick).cuda()
            gl = items[k]["d_leaf"][idx].cpu().numpy()
            gz = items[k]["d_z"][idx].cpu().numpy()
            assert np.abs(gl - rl).max() <= TOL32 * max(np.abs(rl).max(), 1e-300), k
            assert np.abs(gz - rz).max() <= TOL32 * max(np.abs(rz).max(), 1e-300), k
    for e in ens:
        e.close()
