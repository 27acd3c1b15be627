"""Failure detection without a GPU fault: with the test-stall flag every launch of the
recursive step withholds the data of its first block of work, so the kernel's bounded
waits run out (about a millisecond), set the device status word and return.  The host
reads the status, and the context stays usable for a normal plan afterwards."""
import numpy as np
import pytest

import oracle.butterfly as ob
from conftest import rel_l2
from paper_0801_1524_gb300 import native
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "tc"])
def test_bounded_wait_reports_timeout_and_context_survives(prec):
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(2, 64.0, 5, 400, 400, 31)
    f = inst.sources()[0]
    stalled = Plan(inst.x, inst.k, inst.N, inst.p, precision=prec, flags=native.BFLY_FLAG_TEST_STALL)
    stalled.forward(torch.as_tensor(f, device="cuda"))
    bits = stalled.device_status()
    assert bits & 4, bits            # the compute warps gave up waiting for their data
    assert stalled.device_status() == 0   # reading clears the word
    good = Plan(inst.x, inst.k, inst.N, inst.p)
    u = good.forward(torch.as_tensor(f, device="cuda")).cpu().numpy()
    assert good.device_status() == 0
    assert rel_l2(u, ob.butterfly(inst.x, inst.k, f, inst.N, inst.p)) < 1e-6


def test_stream_status_reads_only_its_stream():
    # the status word read in the order of one stream (bfly_stream_status): the stalled
    # launches' bits are seen on the stream they ran on, and reading clears them
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(2, 64.0, 5, 400, 400, 32)
    stalled = Plan(inst.x, inst.k, inst.N, inst.p, flags=native.BFLY_FLAG_TEST_STALL)
    side = torch.cuda.Stream()
    f = torch.as_tensor(inst.sources()[0], device="cuda")
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        stalled.forward(f)
        assert stalled.stream_status(side) & 4
        assert stalled.stream_status(side) == 0
    good = Plan(inst.x, inst.k, inst.N, inst.p)
    good.forward(f)
    assert good.stream_status() == 0


def test_measured_peaks_are_plausible():
    # bfly_measure_peak: FP32 multiply-add loops reach tens of TFLOP/s on this part, the
    # paired form at least as much as the scalar one, FP64 far less
    from paper_0801_1524_gb300.plan import measure_peak
    fp32x2, fp32, fp64 = (measure_peak(k) / 1e12 for k in ("fp32x2", "fp32", "fp64"))
    assert 10.0 < fp32 < 200.0 and 10.0 < fp32x2 < 200.0
    assert fp32x2 > 0.8 * fp32
    assert 0.1 < fp64 < fp32
