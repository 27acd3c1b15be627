"""The recursive step on the tensor cores (precision "tc"): eight right-hand sides of a box
pair per MMA column block, TF32 operands compensated to FP32 accuracy (both operands split
hi + lo, three products), FP32 accumulation.  Same leaf and final steps and the same
chunk programs as the FP32 path, so the results must match the FP32 path and the oracle's
butterfly within the FP32 gate, for any number of right-hand sides (full and partial
groups of eight), forward and adjoint, single plans and batches."""
import numpy as np
import pytest

import oracle.butterfly as ob
from conftest import rel_l2
from paper_0801_1524_gb300 import native
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tol(p):
    return 1e-6 if p <= 7 else 4e-6


@pytest.mark.parametrize("N,p,nrhs", [(64.0, 7, 8), (256.0, 7, 16), (100.5, 7, 11), (128.0, 5, 3),
                                      (32.0, 3, 9), (64.0, 9, 8), (1024.0, 7, 1)])
def test_tc_matches_fp32_and_oracle(N, p, nrhs):
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(2, N, p, 400, 350, 40 + nrhs, edge_fraction=0.2) if N < 1000 else \
        w.Instance("c", 2, N, p, w.sample_curve(w.circle_curve(), N), w.sample_curve(w.star_curve(5), N))
    f = inst.sources(nrhs=nrhs)
    tc = Plan(inst.x, inst.k, N, p, precision="tc", max_nrhs=nrhs)
    assert tc.info()["prec"] == native.BFLY_PREC_TC
    fp32 = Plan(inst.x, inst.k, N, p, precision="fp32", max_nrhs=nrhs)
    ft = torch.as_tensor(f, dtype=torch.complex64, device="cuda")
    u_tc = tc.forward(ft)
    u_32 = fp32.forward(ft)
    assert tc.device_status() == 0
    ref = ob.butterfly(inst.x, inst.k, f, N, p)
    a = u_tc.cpu().numpy().astype(np.complex128)
    b = u_32.cpu().numpy().astype(np.complex128)
    for r in range(nrhs):
        assert rel_l2(a[r], ref[r]) < _tol(p), r
        assert rel_l2(a[r], b[r]) < _tol(p), r
    # right-hand sides are independent: a single one through the same plan is the same
    one = tc.forward(ft[nrhs - 1]).cpu().numpy().astype(np.complex128)
    assert rel_l2(one, a[nrhs - 1]) < 1e-6


@pytest.mark.parametrize("nrhs", [8, 5])
def test_tc_adjoint_is_the_transpose(nrhs):
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(2, 256.0, 7, 900, 800, 50, edge_fraction=0.2)
    P = Plan(inst.x, inst.k, 256.0, 7, precision="tc", max_nrhs=nrhs)
    Q = Plan(inst.x, inst.k, 256.0, 7, precision="fp32", max_nrhs=nrhs)
    f = torch.as_tensor(inst.sources(nrhs=nrhs), dtype=torch.complex64, device="cuda")
    v = torch.as_tensor(w.gaussian_sources(inst.x.shape[0], nrhs=nrhs, seed=9), dtype=torch.complex64,
                        device="cuda")
    u = P.forward(f).cpu().numpy().astype(np.complex128)
    g = P.adjoint(v).cpu().numpy().astype(np.complex128)
    g32 = Q.adjoint(v).cpu().numpy().astype(np.complex128)
    vv, ff = v.cpu().numpy().astype(np.complex128), f.cpu().numpy().astype(np.complex128)
    for r in range(nrhs):
        assert rel_l2(g[r], g32[r]) < 1e-6
        lhs, rhs = np.vdot(vv[r], u[r]), np.vdot(g[r], ff[r])
        assert abs(lhs - rhs) / (np.linalg.norm(u[r]) * np.linalg.norm(vv[r])) < 1e-6


def test_tc_batch_equals_its_plans():
    from paper_0801_1524_gb300.plan import Batch, Plan
    sizes = (64.0, 700.5, 128.0, 300.25)
    insts = []
    for i, N in enumerate(sizes):
        insts.append(w.Instance(f"b{i}", 2, N, 7, w.sample_curve(w.star_curve(2 * i + 1000), N),
                                w.sample_curve(w.star_curve(2 * i + 1001), N), nrhs=16, f_seed=i))
    plans = [Plan(I.x, I.k, I.N, 7, precision="tc", max_nrhs=16) for I in insts]
    fs = [torch.as_tensor(I.sources(), dtype=torch.complex64, device="cuda") for I in insts]
    ref = [P.forward(f) for P, f in zip(plans, fs)]
    batch = Batch(plans)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        us = [torch.empty_like(r) for r in ref]
        for _ in range(2):
            batch.forward(fs, us, stream=side)
    side.synchronize()
    assert batch.device_status() == 0
    for u, r in zip(us, ref):
        assert torch.equal(u, r)
    oracle = ob.butterfly(insts[0].x, insts[0].k, insts[0].sources(), insts[0].N, 7)
    assert rel_l2(us[0].cpu().numpy().astype(np.complex128), oracle) < 1e-6


def test_tc_rejects_3d():
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(3, 8.0, 5, 50, 50, 3)
    with pytest.raises(native.BflyError) as e:
        Plan(inst.x, inst.k, 8.0, 5, precision="tc")
    assert e.value.status == 4
