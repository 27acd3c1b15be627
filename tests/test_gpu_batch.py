"""Batched execution: instances of uneven N (star-shaped curve pairs), several right-hand
sides each, one recursive-step launch per stage over all of them, captured in a CUDA
graph on a side stream and replayed.  Every instance must equal its own plan's forward
transform (the same per-chunk arithmetic) and match the oracle."""
import numpy as np
import pytest

import oracle.butterfly as ob
from conftest import rel_l2
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _instances(sizes=(64.0, 512.0, 128.0, 1024.0, 32.0, 256.0)):
    out = []
    for i, N in enumerate(sizes):
        x = w.sample_curve(w.star_curve(2 * i + 1000), N)
        k = w.sample_curve(w.star_curve(2 * i + 1001), N)
        out.append(w.Instance(f"b{i}", 2, N, 7, x, k, nrhs=3, f_seed=i))
    return out


GENERAL_N = (64.0, 700.5, 128.0, 1000.0, 40.0, 300.25)  # powers of two and not


@pytest.mark.parametrize("sizes", ["pow2", "general"])
@pytest.mark.parametrize("prec,dtype", [("fp32", torch.complex64), ("fp64", torch.complex128)])
def test_batch_matches_plans_and_oracle(prec, dtype, sizes):
    from paper_0801_1524_gb300.plan import Batch, Plan
    insts = _instances() if sizes == "pow2" else _instances(GENERAL_N)
    plans = [Plan(I.x, I.k, I.N, I.p, precision=prec, max_nrhs=3) for I in insts]
    batch = Batch(plans)
    fs = [torch.as_tensor(I.sources(), dtype=dtype, device="cuda") for I in insts]
    ref = [P.forward(f) for P, f in zip(plans, fs)]
    us = batch.forward(fs)  # default stream: direct launches
    torch.cuda.synchronize()
    for u, r in zip(us, ref):
        assert torch.equal(u, r)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        us2 = [torch.empty_like(r) for r in ref]
        for _ in range(3):  # capture, then replays
            batch.forward(fs, us2, stream=side)
    side.synchronize()
    for u, r in zip(us2, ref):
        assert torch.equal(u, r)
    assert batch.device_status() == 0
    tol = 1e-6 if prec == "fp32" else 1e-9
    for I, u in zip(insts[:4], us):
        oracle = ob.butterfly(I.x, I.k, I.sources(), I.N, I.p)
        assert rel_l2(u.cpu().numpy().astype(np.complex128), oracle) < tol


def test_batch_rejects_mixed_plans():
    from paper_0801_1524_gb300.plan import Batch, Plan
    from paper_0801_1524_gb300.native import BflyError
    a = w.small_random(2, 64.0, 7, 100, 100, 1)
    b = w.small_random(2, 64.0, 5, 100, 100, 2)
    with pytest.raises(BflyError):
        Batch([Plan(a.x, a.k, a.N, 7), Plan(b.x, b.k, b.N, 5)])


@pytest.mark.slow
def test_star_batch_full_size():
    # the batched workload as the benchmark runs it: 64 star-curve instances, N drawn
    # log-uniformly in [512, 16384] (not powers of two), p = 7, 16 complex64 right-hand
    # sides each, graph replay on a side stream
    from paper_0801_1524_gb300.plan import Batch, Plan
    insts = w.star_batch(nrhs=16)
    out = {}
    for prec, dtype in (("fp32", torch.complex64), ("tc", torch.complex64), ("fp64", torch.complex128)):
        plans = [Plan(I.x, I.k, I.N, I.p, precision=prec, max_nrhs=16) for I in insts]
        batch = Batch(plans)
        fs = [torch.as_tensor(I.sources(), device="cuda").to(dtype) for I in insts]
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            us = [torch.empty((16, I.x.shape[0]), dtype=dtype, device="cuda") for I in insts]
            for _ in range(2):  # capture, then a replay
                batch.forward(fs, us, stream=side)
        side.synchronize()
        assert batch.device_status() == 0
        if prec != "fp64":
            # every instance equals its own plan's transform (the same chunk arithmetic)
            for P, f, u in zip(plans, fs, us):
                assert torch.equal(u, P.forward(f))
        out[prec] = [u.to(torch.complex128).cpu().numpy() for u in us]
        del batch, plans
    # FP32 (multiply-adds) and the tensor-core path against FP64 on every instance and
    # right-hand side
    for prec in ("fp32", "tc"):
        worst = max(rel_l2(a[r], b[r]) for a, b in zip(out[prec], out["fp64"]) for r in range(16))
        assert worst < 1e-6, (prec, worst)
    # the two smallest instances against the oracle's butterfly, all 16 right-hand sides
    for i in sorted(range(len(insts)), key=lambda i: insts[i].N)[:2]:
        I = insts[i]
        ref = ob.butterfly(I.x, I.k, I.sources(), I.N, I.p)
        assert rel_l2(out["fp64"][i], ref) < 1e-9
        assert rel_l2(out["fp32"][i], ref) < 1e-6
