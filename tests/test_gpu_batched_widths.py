"""The batched persistent forward + adjoint at the merged path widths the
heterogeneous batch spends most of its time on (11-16 unique features), against
the FP64 oracle on every request: phi element-wise (orc_shap_exact) and the
gradients of sum(grad_phi * phi) with respect to leaf values and edge weights
(orc_grad_exact).

Widths 13-16 run two samples per lane (64 per warp) when the request's
64-sample phi tile fits the register class's shared memory (F <= 91 for widths
11-16), otherwise one sample per lane with a shared tile and atomics.  The
requests below cover both sides of that cut (F = 91 and F = 92), a full packed
warp tile (M = 64), a ragged one (M = 65), tiles spread over warps (M = 129)
and over work items (M = 300), F up to 200, and a forward-only request."""
import numpy as np
import pytest

import oracle
import synth
from helpers import caterpillar_ensemble, rel_err_rows

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


def _mixed(seed, cat_depths, F, grown_depth, grown_trees, n_train=4000):
    """Caterpillar trees (every width 1..depth present) plus randomly grown ones."""
    parts = [caterpillar_ensemble(seed, cat_depths, F)]
    if grown_trees:
        parts.append(synth.grow(seed + 1, grown_trees, grown_depth, F, n_train, 0.1, min_rows=5))
    return synth.concat(parts)


# (name, ensemble, M, with_grad)
def _requests():
    reqs = []
    reqs.append(("cat13-16_F40_M64", caterpillar_ensemble(8101, [13, 14, 15, 16, 16, 15, 14, 13], 40), 64, True))
    reqs.append(("mix_F91_M129", _mixed(8102, [16, 15, 14, 13], 91, 16, 3), 129, True))   # packed at the cut
    reqs.append(("mix_F92_M65", _mixed(8103, [13, 14, 15, 16], 92, 14, 3), 65, True))     # one sample per lane
    reqs.append(("grown16_F60_M300", _mixed(8104, [16], 60, 16, 4), 300, True))
    reqs.append(("mix_F200_M129", _mixed(8105, [16, 14], 200, 14, 3), 129, True))        # shared tile, atomics
    reqs.append(("cat13-16_F50_M33_fwd", caterpillar_ensemble(8106, [13, 14, 15, 16], 50), 33, False))
    return reqs


def test_batched_widths_13_to_16_against_the_oracle(qts):
    import torch

    reqs = _requests()
    items, data = [], []
    widths = set()
    for k, (name, ens, M, grad) in enumerate(reqs):
        F = ens.n_features
        X = synth.normal(9100 + k, synth.STREAM_X, (M, F))
        G = synth.normal(9100 + k, synth.STREAM_GRAD, (M, F + 1)) if grad else None
        E = qts.Ensemble.from_arrays(ens)
        widths |= {w for w, n in E.info()["buckets"] if n > 0}
        items.append(dict(ens=E, X=torch.from_numpy(X).cuda(),
                          grad_phi=torch.from_numpy(G).cuda() if grad else None,
                          phi=torch.empty((M, F + 1), dtype=torch.float64, device="cuda"),
                          d_leaf=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda") if grad else None,
                          d_z=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda") if grad else None))
        data.append((name, ens, X, G))
    assert {13, 14, 15, 16} <= widths, widths
    qts.batched_fwd_bwd(qts.make_requests(items))
    torch.cuda.synchronize()
    for (name, ens, X, G), it in zip(data, items):
        it["ens"].sync_status()
        phi = it["phi"].cpu().numpy()
        ref = oracle.shap_exact(ens, X)
        assert rel_err_rows(phi, ref).max() <= TOL32, name
        if G is not None:
            dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
            assert rel(it["d_leaf"].cpu().numpy(), dl_ref) <= TOL32, name
            assert rel(it["d_z"].cpu().numpy(), dz_ref) <= TOL32, name
    for it in items:
        it["ens"].close()


def test_batched_single_request_per_width(qts):
    """One request per width 13..16 alone in a batch (each launches only the
    widths-11-16 class), F = 91, M = 65, against the oracle."""
    import torch

    for D in (13, 14, 15, 16):
        ens = caterpillar_ensemble(8200 + D, [D] * 6, 91)
        F, M = 91, 65
        X = synth.normal(8200 + D, synth.STREAM_X, (M, F))
        G = synth.normal(8200 + D, synth.STREAM_GRAD, (M, F + 1))
        E = qts.Ensemble.from_arrays(ens)
        it = dict(ens=E, X=torch.from_numpy(X).cuda(), grad_phi=torch.from_numpy(G).cuda(),
                  phi=torch.empty((M, F + 1), dtype=torch.float64, device="cuda"),
                  d_leaf=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda"),
                  d_z=torch.empty(E.n_nodes, dtype=torch.float64, device="cuda"))
        qts.batched_fwd_bwd(qts.make_requests([it]))
        torch.cuda.synchronize()
        E.sync_status()
        assert rel_err_rows(it["phi"].cpu().numpy(), oracle.shap_exact(ens, X)).max() <= TOL32, D
        dl_ref, dz_ref = oracle.grad_exact(ens, X, G)
        assert rel(it["d_leaf"].cpu().numpy(), dl_ref) <= TOL32, D
        assert rel(it["d_z"].cpu().numpy(), dz_ref) <= TOL32, D
        E.close()
