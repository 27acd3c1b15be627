"""The recursive step on groups of eight right-hand sides with paired FP32 multiply-adds
(BFLY_FLAG_RHS_GROUPS, precision "fp32g"): the same operators, applied to every fibre in
the same order as the default FP32 kernel, so the transform must equal the default FP32
transform bit for bit, for full and partial groups, forward and adjoint, single plans and
batches; and the oracle's butterfly within the FP32 gate."""
import numpy as np
import pytest

import oracle.butterfly as ob
from conftest import rel_l2
from paper_0801_1524_gb300 import native
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,p,nrhs", [(256.0, 7, 16), (100.5, 7, 11), (128.0, 5, 3), (64.0, 9, 8),
                                      (32.0, 3, 1), (2048.0, 7, 8)])
def test_groups_equal_the_default_kernel(N, p, nrhs):
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(2, N, p, 500, 450, 70 + nrhs, edge_fraction=0.2) if N < 1000 else \
        w.Instance("c", 2, N, p, w.sample_curve(w.circle_curve(), N), w.sample_curve(w.star_curve(8), N))
    f = torch.as_tensor(inst.sources(nrhs=nrhs), dtype=torch.complex64, device="cuda")
    G = Plan(inst.x, inst.k, N, p, precision="fp32g", max_nrhs=nrhs)
    assert G.info()["rhs_groups"] == 1
    F = Plan(inst.x, inst.k, N, p, precision="fp32", max_nrhs=nrhs)
    ug, uf = G.forward(f), F.forward(f)
    assert G.device_status() == 0
    assert torch.equal(ug, uf)
    v = torch.as_tensor(w.gaussian_sources(inst.x.shape[0], nrhs=nrhs, seed=3), dtype=torch.complex64,
                        device="cuda")
    assert torch.equal(G.adjoint(v), F.adjoint(v))
    if N < 1000:
        ref = ob.butterfly(inst.x, inst.k, inst.sources(nrhs=nrhs), N, p)
        got = ug.cpu().numpy().astype(np.complex128)
        for r in range(nrhs):
            assert rel_l2(got[r], ref[r]) < (1e-6 if p <= 7 else 4e-6)


def test_groups_batch_and_mixing_rejected():
    from paper_0801_1524_gb300.plan import Batch, Plan
    insts = [w.Instance(f"b{i}", 2, N, 7, w.sample_curve(w.star_curve(2 * i + 1000), N),
                        w.sample_curve(w.star_curve(2 * i + 1001), N), nrhs=16, f_seed=i)
             for i, N in enumerate((64.0, 700.5, 300.25))]
    fs = [torch.as_tensor(I.sources(), dtype=torch.complex64, device="cuda") for I in insts]
    G = [Plan(I.x, I.k, I.N, 7, precision="fp32g", max_nrhs=16) for I in insts]
    F = [Plan(I.x, I.k, I.N, 7, precision="fp32", max_nrhs=16) for I in insts]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ug = Batch(G).forward(fs, stream=side)
        uf = [P.forward(f, stream=side) for P, f in zip(F, fs)]
    side.synchronize()
    for a, b in zip(ug, uf):
        assert torch.equal(a, b)
    with pytest.raises(native.BflyError):
        Batch([G[0], F[1]])


def test_groups_failure_hook():
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(2, 64.0, 5, 400, 400, 31)
    stalled = Plan(inst.x, inst.k, inst.N, inst.p, precision="fp32g", max_nrhs=8,
                   flags=native.BFLY_FLAG_TEST_STALL)
    stalled.forward(torch.as_tensor(inst.sources(nrhs=8), dtype=torch.complex64, device="cuda"))
    assert stalled.device_status() & 4
    assert stalled.device_status() == 0
