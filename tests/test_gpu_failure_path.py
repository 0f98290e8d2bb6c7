"""The device failure path, without a GPU fault: a bounded wait that nothing
completes runs out after about a second, the kernel latches QTS_ERR_TIMEOUT in
the ensemble's status word and returns, the host reads the code, and the
context keeps working."""
import time

import numpy as np
import pytest

import oracle
import synth
from helpers import rel_err_rows

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


def test_bounded_wait_reports_timeout_and_context_survives(qts):
    import torch

    w = synth.workload("small-depth4")
    E = qts.Ensemble.from_arrays(w.ens)
    X = torch.from_numpy(w.X).cuda()
    E.sync_status()
    t0 = time.time()
    E.selftest_wait_timeout()
    with pytest.raises(qts.QtsError) as ei:
        E.sync_status()
    elapsed = time.time() - t0
    assert ei.value.status == 5  # QTS_ERR_TIMEOUT
    assert 0.5 < elapsed < 30.0, elapsed
    E.sync_status()  # the code was read and cleared
    phi = qts.shap_values(E, X).cpu().numpy()
    E.sync_status()
    assert rel_err_rows(phi, oracle.shap_exact(w.ens, w.X)).max() <= 1e-5
    E.close()
