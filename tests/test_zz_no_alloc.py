"""qts_shap_interactions_noalloc: the allocation-free entry point for callers
that may not allocate device memory during a call (graph capture that forbids
allocation nodes, a fixed memory budget owned by another allocator, or code
that cannot absorb cudaMalloc's implicit synchronisation).

Every call clears and reuses one fixed device array shared by the whole
process, so these tests check the results against the FP64 oracle (not only
against the sibling entry point, which runs the same kernels) after calls that
left other sums in that array: a larger call before a small one, a call that
fills the array exactly, and its one-sample-larger neighbour, which must be
refused.

This file is collected last on purpose: it also runs after every other test
has used the library in the same process."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
LIMIT = 2 * 1024 * 1024  # accumulator doubles in the fixed array


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


def _noalloc(q, E, X, out):
    """One call through the C ABI; returns the status."""
    import torch

    M, F = X.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return q.lib().qts_shap_interactions_noalloc(E.handle, ctypes.c_void_p(X.data_ptr()), M, F, 8,
                                                 ctypes.c_void_p(out.data_ptr()), stream)


def _run(q, E, Xh):
    import torch

    X = torch.from_numpy(np.ascontiguousarray(Xh, np.float32)).cuda()
    M, F = X.shape
    out = torch.full((M, F + 1, F + 1), float("nan"), dtype=torch.float32, device="cuda")
    st = _noalloc(q, E, X, out)
    assert st == 0, q.lib().qts_last_error()
    E.sync_status()
    return out.cpu().numpy().astype(np.float64)


def _check_oracle(got, ens, X):
    sii, phi = oracle.sii_exact(ens, X)
    ref = oracle.interaction_matrix(sii, phi)
    scale = np.maximum(np.abs(phi.sum(1)), np.abs(phi[:, :-1]).max(1))
    err = np.abs(got - ref).reshape(len(X), -1).max(1) / scale
    assert err.max() <= TOL32, err.max()
    F = X.shape[1]
    rows = got[:, :F, :F].sum(axis=2)  # interaction rows sum to phi_i
    assert (np.abs(rows - phi[:, :F]).max(1) / scale).max() <= TOL32


def test_noalloc_matches_workspace_entry_point_twice(qts):
    import torch

    w = synth.workload("pairs-depth6", n_samples=300, n_trees=60)
    E = qts.Ensemble.from_arrays(w.ens)
    X = torch.from_numpy(w.X).cuda()
    M, F = w.X.shape
    ref = qts.shap_interactions(E, X).cpu().numpy().astype(np.float64)
    for call in range(2):
        out = torch.full((M, F + 1, F + 1), float("nan"), dtype=torch.float32, device="cuda")
        st = _noalloc(qts, E, X, out)
        assert st == 0, qts.lib().qts_last_error()
        E.sync_status()
        got = out.cpu().numpy().astype(np.float64)
        err = np.abs(got - ref).reshape(M, -1).max(axis=1) / _scale(ref)
        assert err.max() <= 1e-5, (call, err.max())
    E.close()


def test_noalloc_small_call_after_a_larger_one_matches_the_oracle(qts):
    big = synth.workload("pairs-depth6", n_samples=4000, n_trees=30)  # (435 + 30) * 4000 doubles
    assert (30 * 29 // 2 + 30) * 4000 <= LIMIT
    E = qts.Ensemble.from_arrays(big.ens)
    _run(qts, E, big.X)  # leaves its sums in the array
    E.close()
    small = synth.workload("pairs-depth6", n_samples=40, n_trees=25)
    E = qts.Ensemble.from_arrays(small.ens)
    got = _run(qts, E, small.X)
    _check_oracle(got, small.ens, small.X)
    E.close()


def test_noalloc_exact_limit_and_its_neighbour(qts):
    """F = 1: (F(F-1)/2 + F) * M = M, so M = 2,097,152 fills the array exactly
    (accepted) and M + 1 is refused; a small call afterwards still matches."""
    import torch

    ens = synth.grow(7301, 6, 5, 1, 4000, 1.0, min_rows=2)
    E = qts.Ensemble.from_arrays(ens)
    Xh = synth.normal(7301, synth.STREAM_X, (LIMIT, 1))
    got = _run(qts, E, Xh)
    # every row: off-diagonals 0, E[f] at [1, 1]; sampled rows against the oracle
    assert np.all(got[:, 0, 1] == 0) and np.all(got[:, 1, 0] == 0)
    rows = np.r_[0:16, LIMIT // 2:LIMIT // 2 + 16, LIMIT - 16:LIMIT]
    _check_oracle(got[rows], ens, Xh[rows])
    # and every row against the workspace entry point
    ref = qts.shap_interactions(E, torch.from_numpy(Xh).cuda()).cpu().numpy().astype(np.float64)
    err = np.abs(got - ref).reshape(LIMIT, -1).max(axis=1) / _scale(ref)
    assert err.max() <= TOL32, err.max()
    del ref

    X1 = torch.zeros((LIMIT + 1, 1), dtype=torch.float32, device="cuda")
    out1 = torch.empty((1,), dtype=torch.float32, device="cuda")
    assert _noalloc(qts, E, X1, out1) == 4  # QTS_ERR_UNSUPPORTED
    assert b"fixed scratch" in qts.lib().qts_last_error()
    del X1

    small = Xh[:100]
    _check_oracle(_run(qts, E, small), ens, small)
    E.close()


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch(qts):
    import torch

    w = synth.workload("pairs-depth6", n_samples=8, n_trees=4)
    E = qts.Ensemble.from_arrays(w.ens)
    F = w.X.shape[1]
    M = 5000  # (F(F-1)/2 + F) * M = 465 * 5000 > 2,097,152
    X = torch.zeros((M, F), dtype=torch.float32, device="cuda")
    out = torch.empty((1,), dtype=torch.float32, device="cuda")
    st = _noalloc(qts, E, X, out)
    assert st == 4  # QTS_ERR_UNSUPPORTED
    assert b"fixed scratch" in qts.lib().qts_last_error()
    E.close()
