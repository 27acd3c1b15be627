"""The split sweep on the GPU (bfly_execute_to_stage / bfly_execute_from_stage) and the
sharded transform built on it (paper_0801_1524_gb300/sharded.py), its ranks run one after
the other in this process on one GPU with the exchange done in memory (the kernels of
one rank never wait for another's).  Every rank's potentials must equal the unsharded
transform's for its targets, and the oracle's butterfly."""
import numpy as np
import pytest

import oracle.butterfly as ob
from conftest import rel_l2
from paper_0801_1524_gb300 import native
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_split_at_every_boundary_is_the_transform(prec):
    from paper_0801_1524_gb300.plan import Plan
    inst = w.small_random(2, 512.0, 7, 900, 800, 61, edge_fraction=0.2)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    P = Plan(inst.x, inst.k, inst.N, inst.p, precision=prec, max_nrhs=2)
    f = torch.as_tensor(inst.sources(nrhs=2), dtype=dt, device="cuda")
    ref = P.forward(f)
    v = torch.as_tensor(w.gaussian_sources(inst.x.shape[0], nrhs=2, seed=62), dtype=dt, device="cuda")
    ref_adj = P.adjoint(v)
    for t in P.boundaries():
        c = P.to_stage(f, t)
        u = P.from_stage(c, t)
        ca = P.to_stage(v, t, adjoint=True)
        g = P.from_stage(ca, t, adjoint=True)
        torch.cuda.synchronize()
        assert torch.equal(u, ref), t
        assert torch.equal(g, ref_adj), t
    inner = [t for t in range(P.info()["L"] + 1) if t not in P.boundaries()]
    if inner:
        with pytest.raises(native.BflyError):
            P.to_stage(f, inner[0])


@pytest.mark.parametrize("world,prec,N,p", [(2, "fp32", 2048.0, 7), (4, "fp64", 1000.5, 5), (3, "fp32", 4096.0, 5)])
def test_sharded_ranks_equal_the_unsharded_transform(world, prec, N, p):
    from paper_0801_1524_gb300 import sharded
    from paper_0801_1524_gb300.plan import Plan
    x = w.sample_curve(w.circle_curve(), N)
    k = w.sample_curve(w.star_curve(4), N)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    f = w.gaussian_sources(k.shape[0], nrhs=2, seed=2)
    lay = sharded.ShardLayout(x, k, N, p, world)
    ranks = [sharded.ShardedTransform(lay, r, precision=prec, max_nrhs=2) for r in range(world)]
    ups = [R.upper(torch.as_tensor(f[:, lay.sources[r]], dtype=dt, device="cuda")) for r, R in enumerate(ranks)]
    packed = [sharded.pack(lay, r, c) for r, c in enumerate(ups)]
    full = Plan(x, k, N, p, precision=prec, max_nrhs=2).forward(torch.as_tensor(f, dtype=dt, device="cuda"))
    full = full.cpu().numpy().astype(np.complex128)
    oracle = ob.butterfly(x, k, f, N, p) if N <= 2048 else None
    tol = 2e-6 if prec == "fp32" else 1e-12
    for r, R in enumerate(ranks):
        u = R.lower(sharded.assemble(lay, r, [packed[q][r] for q in range(world)]))
        torch.cuda.synchronize()
        u = u.cpu().numpy().astype(np.complex128)
        tgt = lay.targets[r]
        assert len(tgt) > 0
        for j in range(2):
            assert rel_l2(u[j], full[j, tgt]) < tol
            if oracle is not None:
                assert rel_l2(u[j], oracle[j, tgt]) < (1e-6 if prec == "fp32" else 1e-9)


@pytest.mark.parametrize("world,prec", [(2, "fp32"), (3, "fp64")])
def test_sharded_adjoint_is_the_transpose(world, prec):
    from paper_0801_1524_gb300 import sharded
    from paper_0801_1524_gb300.plan import Plan
    N, p = 2048.0, 7
    x = w.sample_curve(w.circle_curve(), N)
    k = w.sample_curve(w.star_curve(6), N)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    v = w.gaussian_sources(x.shape[0], nrhs=2, seed=7)
    lay = sharded.ShardLayout(x, k, N, p, world)
    ranks = [sharded.ShardedTransform(lay, r, precision=prec, max_nrhs=2) for r in range(world)]
    ups = [R.upper_adjoint(torch.as_tensor(v[:, lay.targets[r]], dtype=dt, device="cuda"))
           for r, R in enumerate(ranks)]
    packed = [sharded.pack_adjoint(lay, r, c) for r, c in enumerate(ups)]
    full = Plan(x, k, N, p, precision=prec, max_nrhs=2).adjoint(torch.as_tensor(v, dtype=dt, device="cuda"))
    full = full.cpu().numpy().astype(np.complex128)
    tol = 2e-6 if prec == "fp32" else 1e-12
    for r, R in enumerate(ranks):
        g = R.lower_adjoint(sharded.assemble_adjoint(lay, r, [packed[q][r] for q in range(world)]))
        torch.cuda.synchronize()
        g = g.cpu().numpy().astype(np.complex128)
        src = lay.sources[r]
        for j in range(2):
            assert rel_l2(g[j], full[j, src]) < tol
