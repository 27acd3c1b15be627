"""The single-launch sweep (BFLY_FLAG_DATAFLOW): the chunks of every step of the recursive
step (Sec. 2.2 step 3) in one launch, each started once the chunks whose outputs it reads
have published them.  Every chunk runs the same program on the same inputs as in the
step-by-step launches, so the results must be bit-identical to those, forward and
adjoint, in both precisions, in 2D and 3D, for one and several right-hand sides, over
repeated launches (the per-chunk flags carry the launch's epoch) and with launches of
other plans and directions queued behind one another, and match the oracle."""
import numpy as np
import pytest

import oracle.butterfly as ob
from conftest import rel_l2
from paper_0801_1524_gb300 import native
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(inst, prec, nrhs, **kw):
    # the same steps launched one by one (a) and in one launch (b)
    from paper_0801_1524_gb300.plan import Plan
    b = Plan(inst.x, inst.k, inst.N, inst.p, precision=prec, max_nrhs=nrhs, dataflow=True, **kw)
    a = Plan(inst.x, inst.k, inst.N, inst.p, precision=prec, max_nrhs=nrhs,
             stages=b.info()["stages_per_launch"], **kw)
    assert b.info()["dataflow"] == 1 and a.info()["dataflow"] == 0
    assert a.steps() == b.steps()
    return a, b


CASES = [
    # (dim, N, p, nx, nk, seed): trees from two steps of a few chunks (fewer than the blocks
    # of the grid) to six steps of thousands of chunks
    (2, 16.0, 5, 200, 150, 1),
    (2, 100.5, 7, 600, 500, 2),
    (2, 512.0, 7, 1500, 1400, 3),
    (3, 8.0, 5, 400, 300, 4),
    (3, 16.0, 3, 800, 700, 5),
]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("case", CASES)
def test_bit_identical_to_step_by_step(case, prec):
    dim, N, p, nx, nk, seed = case
    inst = w.small_random(dim, N, p, nx, nk, seed, edge_fraction=0.2)
    a, b = _pair(inst, prec, 3)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    for nrhs in (1, 3):
        f = torch.as_tensor(inst.sources(nrhs=nrhs), dtype=dt, device="cuda")
        v = torch.as_tensor(w.gaussian_sources(inst.x.shape[0], nrhs=nrhs, seed=seed + 50), dtype=dt,
                            device="cuda")
        ref_f, ref_a = a.forward(f), a.adjoint(v)
        for _ in range(3):  # repeated launches, each with its own epoch, queued back to back
            u, g = b.forward(f), b.adjoint(v)
            torch.cuda.synchronize()
            assert torch.equal(u, ref_f)
            assert torch.equal(g, ref_a)
    assert b.device_status() == 0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_curve_matches_oracle_and_step_by_step(prec):
    from paper_0801_1524_gb300.plan import Plan
    x = w.sample_curve(w.circle_curve(), 2048.0)
    k = w.sample_curve(w.star_curve(3), 2048.0)
    b = Plan(x, k, 2048.0, 7, precision=prec, max_nrhs=2, dataflow=True)
    a = Plan(x, k, 2048.0, 7, precision=prec, max_nrhs=2, stages=b.info()["stages_per_launch"])
    assert b.info()["stages_per_launch"] == 2 and a.steps() == b.steps()
    f = w.gaussian_sources(k.shape[0], nrhs=2, seed=9)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    ft = torch.as_tensor(f, dtype=dt, device="cuda")
    u = b.forward(ft)
    assert torch.equal(u, a.forward(ft))
    ref = ob.butterfly(x, k, f, 2048.0, 7)
    got = u.cpu().numpy().astype(np.complex128)
    tol = 1e-6 if prec == "fp32" else 1e-9
    for j in range(2):
        assert rel_l2(got[j], ref[j]) < tol
    assert b.device_status() == 0


def test_alternating_plans_directions_and_sizes():
    # two dataflow plans and both directions interleaved on one stream, the right-hand
    # side count changing between launches
    inst1 = w.small_random(2, 256.0, 7, 900, 800, 11)
    inst2 = w.small_random(2, 300.0, 5, 700, 900, 12)
    a1, b1 = _pair(inst1, "fp32", 4)
    a2, b2 = _pair(inst2, "fp32", 4)
    for nrhs in (2, 4, 1, 3):
        f1 = torch.as_tensor(inst1.sources(nrhs=nrhs, dtype=np.complex64), device="cuda")
        f2 = torch.as_tensor(inst2.sources(nrhs=nrhs, dtype=np.complex64), device="cuda")
        v2 = torch.as_tensor(w.gaussian_sources(inst2.x.shape[0], nrhs=nrhs, seed=nrhs, dtype=np.complex64),
                             device="cuda")
        outs = [b1.forward(f1), b2.adjoint(v2), b2.forward(f2), b1.forward(f1)]
        refs = [a1.forward(f1), a2.adjoint(v2), a2.forward(f2), a1.forward(f1)]
        torch.cuda.synchronize()
        for o, r in zip(outs, refs):
            assert torch.equal(o, r)
    assert b1.device_status() == 0 and b2.device_status() == 0


def test_events_and_host_buffers():
    inst = w.small_random(2, 1024.0, 7, 2500, 2400, 21)
    a, b = _pair(inst, "fp32", 1)
    f = inst.sources(dtype=np.complex64)
    ref = a.forward(torch.as_tensor(f, device="cuda")).cpu().numpy()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(b.info()["steps"] + 3)]
    for e in ev:
        e.record()
    u = b.with_events(torch.as_tensor(f, device="cuda"), ev)
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy(), ref)
    assert ev[0].elapsed_time(ev[-1]) > 0
    host = b.execute_host(f)
    assert np.array_equal(host.reshape(ref.shape), ref)


def test_stalled_dataflow_launch_reports_and_context_survives():
    # the test-stall hook withholds each block's first chunk: its compute warps, and the
    # blocks that wait for its outputs, give up their bounded waits and the launch returns
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(2, 256.0, 5, 800, 800, 31)
    f = torch.as_tensor(inst.sources(), device="cuda")
    stalled = Plan(inst.x, inst.k, inst.N, inst.p, dataflow=True, flags=native.BFLY_FLAG_TEST_STALL)
    stalled.forward(f)
    bits = stalled.device_status()
    assert bits & 4, bits
    good = Plan(inst.x, inst.k, inst.N, inst.p, dataflow=True)
    u = good.forward(f).cpu().numpy()
    assert good.device_status() == 0
    assert rel_l2(u, ob.butterfly(inst.x, inst.k, inst.sources()[0], inst.N, inst.p)) < 1e-6


def test_unsupported_with_tensor_cores_and_groups():
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(2, 64.0, 7, 300, 300, 41)
    for prec in ("tc", "fp32g"):
        with pytest.raises(native.BflyError):
            Plan(inst.x, inst.k, inst.N, inst.p, precision=prec, max_nrhs=8, dataflow=True)
