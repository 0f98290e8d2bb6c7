"""qts_shap_interactions_noalloc: the allocation-free entry point for callers
that may not allocate device memory during a call (graph capture that forbids
allocation nodes, a fixed memory budget owned by another allocator, or code
that cannot absorb cudaMalloc's implicit synchronisation).  It must give the
same matrices as qts_shap_interactions, call after call, since every call
reuses (and first clears) the same fixed device array.

This file is collected last on purpose: it also runs after every other test
has used the library in the same process."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qts():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_04497_gb300 import build as b

    b.build()
    import paper_2605_04497_gb300 as q

    return q


def _scale(ref):
    # per-sample normaliser of the interaction parity tests: max(|f(x)|, max |phi_i|)
    phi = ref.sum(axis=2)
    return np.maximum(np.abs(phi.sum(axis=1)), np.abs(phi[:, :-1]).max(axis=1))


def test_noalloc_matches_workspace_entry_point_twice(qts):
    import torch

    w = synth.workload("pairs-depth6", n_samples=300, n_trees=60)
    E = qts.Ensemble.from_arrays(w.ens)
    X = torch.from_numpy(w.X).cuda()
    M, F = w.X.shape
    ref = qts.shap_interactions(E, X).cpu().numpy().astype(np.float64)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full((M, F + 1, F + 1), float("nan"), dtype=torch.float32, device="cuda")
        st = qts.lib().qts_shap_interactions_noalloc(E.handle, ctypes.c_void_p(X.data_ptr()), M, F, 8,
                                                     ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, qts.lib().qts_last_error()
        E.sync_status()
        got = out.cpu().numpy().astype(np.float64)
        err = np.abs(got - ref).reshape(M, -1).max(axis=1) / _scale(ref)
        assert err.max() <= 1e-5, (call, err.max())
    E.close()


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch(qts):
    import torch

    w = synth.workload("pairs-depth6", n_samples=8, n_trees=4)
    E = qts.Ensemble.from_arrays(w.ens)
    F = w.X.shape[1]
    M = 5000  # (F(F-1)/2 + F) * M = 465 * 5000 > 2,097,152
    X = torch.zeros((M, F), dtype=torch.float32, device="cuda")
    out = torch.empty((1,), dtype=torch.float32, device="cuda")
    st = qts.lib().qts_shap_interactions_noalloc(E.handle, ctypes.c_void_p(X.data_ptr()), M, F, 8,
                                                 ctypes.c_void_p(out.data_ptr()), None)
    assert st == 4  # QTS_ERR_UNSUPPORTED
    assert b"fixed scratch" in qts.lib().qts_last_error()
    E.close()
