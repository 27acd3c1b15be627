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


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(2, 64.0, 5, 400, 400, 31)
    f = inst.sources()[0]
    stalled = Plan(inst.x, inst.k, inst.N, inst.p, flags=native.BFLY_FLAG_TEST_STALL)
    stalled.forward(torch.as_tensor(f, device="cuda"))
    bits = stalled.device_status()
    assert bits & 4, bits            # the compute warps gave up waiting for their data
    assert stalled.device_status() == 0   # reading clears the word
    good = Plan(inst.x, inst.k, inst.N, inst.p)
    u = good.forward(torch.as_tensor(f, device="cuda")).cpu().numpy()
    assert good.device_status() == 0
    assert rel_l2(u, ob.butterfly(inst.x, inst.k, f, inst.N, inst.p)) < 1e-6
