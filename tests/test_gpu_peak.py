"""The FP32-pipe probe (qts_fp32_pipe_peak) against the peak derived from the
device's unit counts: SMs x 128 FP32 lanes x the maximum SM clock.  Packed
f32x2 FMAs must not exceed that derived lane rate (each one occupies the pipe
for two lanes' worth), and independent chains at full occupancy must come
close to it under either form."""
import subprocess

import pytest

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


def _derived_peak():
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                         capture_output=True, text=True)
    mhz = float(out.stdout.strip().splitlines()[0]) if out.returncode == 0 and out.stdout.strip() else 2070.0
    return sms * 128 * mhz * 1e6


def test_probe_against_derived_peak(qts):
    peak = _derived_peak()
    packed = qts.fp32_pipe_peak(True)
    scalar = qts.fp32_pipe_peak(False)
    print(f"derived {peak / 1e12:.2f}, packed {packed / 1e12:.2f}, scalar {scalar / 1e12:.2f} T lane-FMA/s")
    for v in (packed, scalar):
        assert 0.6 * peak <= v <= 1.08 * peak, (v, peak)
