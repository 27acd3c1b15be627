"""The sharded sweep (paper_0801_1524_gb300/sharded.py) on CPU: two gloo ranks, one process
each.  Each rank takes its sources' stage-L charges (the oracle's, Sec. 2.2 step 2),
runs its plan's recursive-step programs down to the middle stage (the library's compiled
chunk programs, executed by the numpy interpreter of test_step_programs with the
operators of the method), exchanges the middle stage with the other rank through the
module's pack / exchange_p2p / assemble, runs the rest of the sweep for its targets, and
must reproduce the stage-0 charges of the unsharded sweep for its targets' leaves.  The
adjoint runs backwards the same way (the conjugate-transposed operators on the adjoint
programs, the exchange transposed by pack_adjoint / assemble_adjoint) and must reproduce
the unsharded adjoint sweep's stage-L charges for each rank's source leaves.  The
partition itself is checked too: every point on exactly one rank, each rank's boxes a
contiguous run of the Morton order."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_steps(P, x, ops, first, last):
    """The plan's forward launches first .. last - 1 on the tiles x (interpreter)."""
    import test_step_programs as tsp
    pairs = {t: a * b for t, a, b in P.stages()}
    steps = P.steps()
    for s in range(first, last):
        t, lev = steps[s]
        x = tsp.run_program(P.program(s), P.dim, P.p, x, pairs[t - lev + 1], ops)
    return x


def _boundary(P, t):
    return P.boundaries().index(t)


def _stage_L_tiles(x, k, f, N, p, P):
    import oracle.butterfly as ob
    import test_step_programs as tsp
    TX, TK, L, F = ob.stage_charges(x, k, f, N, p)
    return tsp._to_plan_order(tsp._rescale(F[L], TX.boxes[0], p), TX.boxes[0], TK.boxes[L], P, L, L)


def _rank(rank, world, port, case, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, HERE)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import test_step_programs as tsp
    from paper_0801_1524_gb300 import sharded
    from paper_0801_1524_gb300 import workloads as w
    from paper_0801_1524_gb300.plan import Plan
    dim, N, p, nx, nk, seed, stages = case
    inst = w.small_random(dim, N, p, nx, nk, seed, edge_fraction=0.2)
    f = inst.sources()[0].astype(np.complex128)
    ops = tsp._method_ops(p)
    lay = sharded.ShardLayout(inst.x, inst.k, N, p, world, stages=stages)
    pd = p ** dim
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # first part: this rank's sources, stage L -> t_mid
        src = lay.sources[rank]
        up = Plan(inst.x, inst.k[src], N, p, host_only=True, stages=stages)
        if len(src):
            gL = _stage_L_tiles(inst.x, inst.k[src], f[src], N, p, up)
            c = _run_steps(up, gL, ops, 0, _boundary(up, lay.t_mid))
        else:
            c = np.zeros((0,) + (p,) * dim, dtype=np.complex128)
        c = torch.as_tensor(c.reshape(1, len(lay.xboxes), lay.n_kboxes(rank), pd))
        sends = [torch.view_as_real(b) for b in sharded.pack(lay, rank, c)]
        shapes = [(1, lay.n_xboxes(rank), lay.n_kboxes(q), pd, 2) for q in range(world)]
        got = sharded.exchange_p2p(sends, shapes, rank, world, dist)
        cin = sharded.assemble(lay, rank, [torch.view_as_complex(g.contiguous()) for g in got])
        # second part: this rank's targets, t_mid -> 0
        lo = Plan(inst.x[lay.targets[rank]], inst.k, N, p, host_only=True, stages=stages)
        g0 = _run_steps(lo, cin.numpy().reshape((-1,) + (p,) * dim), ops, _boundary(lo, lay.t_mid),
                        len(lo.steps()))
        leaves = lo.boxes("x", lay.L)
        dist.barrier()
    finally:
        dist.destroy_process_group()
    out.put((rank, g0, leaves, lay.t_mid, [len(s) for s in lay.sources], [len(t) for t in lay.targets]))


def _run_steps_adjoint(P, x, opsH, first, last):
    """The plan's adjoint launches first - 1, .., last on the tiles x (interpreter)."""
    import test_step_programs as tsp
    pairs = {t: a * b for t, a, b in P.stages()}
    steps = P.steps()
    for s in range(first - 1, last - 1, -1):
        t, lev = steps[s]
        x = tsp.run_program(P.program(s, True), P.dim, P.p, x, pairs[t + 1], opsH)
    return x


def _stage0_tiles(P, L, seed, shape):
    """Seeded stage-0 tiles (T_X leaves x the T_K root) in the order of P's T_X leaves,
    drawn per leaf box so that every plan of a subset of the targets sees the same tile."""
    out = []
    for b in P.boxes("x", L):
        rng = np.random.default_rng([seed] + [int(v) for v in b])
        out.append(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    return np.array(out).reshape((-1,) + shape)


def _rank_adjoint(rank, world, port, case, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, HERE)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import test_step_programs as tsp
    from paper_0801_1524_gb300 import sharded
    from paper_0801_1524_gb300 import workloads as w
    from paper_0801_1524_gb300.plan import Plan
    dim, N, p, nx, nk, seed, stages = case
    inst = w.small_random(dim, N, p, nx, nk, seed, edge_fraction=0.2)
    opsH = np.conj(np.transpose(tsp._method_ops(p), (0, 2, 1)))
    lay = sharded.ShardLayout(inst.x, inst.k, N, p, world, stages=stages)
    pd = p ** dim
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # first part of the adjoint: this rank's targets, stage 0 -> t_mid
        lo = Plan(inst.x[lay.targets[rank]], inst.k, N, p, host_only=True, stages=stages)
        g0 = _stage0_tiles(lo, lay.L, 99, (p,) * dim)
        c = _run_steps_adjoint(lo, g0, opsH, len(lo.steps()), lo.boundaries().index(lay.t_mid))
        c = torch.as_tensor(c.reshape(1, lay.n_xboxes(rank), len(lay.kboxes), pd))
        sends = [torch.view_as_real(b) for b in sharded.pack_adjoint(lay, rank, c)]
        shapes = [(1, lay.n_xboxes(q), lay.n_kboxes(rank), pd, 2) for q in range(world)]
        got = sharded.exchange_p2p(sends, shapes, rank, world, dist)
        cin = sharded.assemble_adjoint(lay, rank, [torch.view_as_complex(g.contiguous()) for g in got])
        # second part: this rank's sources, t_mid -> stage L
        up = Plan(inst.x, inst.k[lay.sources[rank]], N, p, host_only=True, stages=stages)
        gL = _run_steps_adjoint(up, cin.numpy().reshape((-1,) + (p,) * dim), opsH, up.boundaries().index(lay.t_mid), 0)
        leaves = up.boxes("k", lay.L)
        dist.barrier()
    finally:
        dist.destroy_process_group()
    out.put((rank, gL, leaves))


CASES = [(2, 128.0, 5, 500, 400, 1, 0), (2, 200.5, 7, 400, 350, 2, 0), (2, 256.0, 5, 600, 500, 3, 1),
         (3, 16.0, 3, 300, 260, 4, 0)]


@pytest.mark.parametrize("case", CASES)
def test_two_gloo_ranks_reproduce_the_unsharded_sweep(case):
    sys.path.insert(0, HERE)
    import test_step_programs as tsp
    from paper_0801_1524_gb300 import workloads as w
    from paper_0801_1524_gb300.plan import Plan
    dim, N, p, nx, nk, seed, stages = case
    world = 2
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda v: v[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    # the unsharded sweep of all points
    inst = w.small_random(dim, N, p, nx, nk, seed, edge_fraction=0.2)
    f = inst.sources()[0].astype(np.complex128)
    P = Plan(inst.x, inst.k, N, p, host_only=True, stages=stages)
    ref = tsp.sweep(P, _stage_L_tiles(inst.x, inst.k, f, N, p, P), tsp._method_ops(p))
    L = P.info()["L"]
    row = {tuple(b): i for i, b in enumerate(P.boxes("x", L))}
    scale = np.abs(ref).max()
    seen = set()
    for rank, g0, leaves, t_mid, nsrc, ntgt in res:
        assert 0 < t_mid < L or L <= 1
        assert sum(nsrc) == nk and sum(ntgt) == nx
        assert min(nsrc) > 0 and min(ntgt) > 0           # both ranks have work
        idx = np.array([row[tuple(b)] for b in leaves])
        assert not seen & set(idx.tolist())
        seen |= set(idx.tolist())
        err = np.abs(g0 - ref[idx]).max() / scale
        assert err < 1e-12, (rank, err)
    assert seen == set(range(len(row)))                # every target leaf on one rank


def test_layout_partitions_points_into_contiguous_runs():
    sys.path.insert(0, ROOT)
    from paper_0801_1524_gb300 import sharded
    from paper_0801_1524_gb300 import workloads as w
    inst = w.star32768()
    for world in (2, 4, 8):
        lay = sharded.ShardLayout(inst.x, inst.k, inst.N, inst.p, world)
        assert sorted(np.concatenate(lay.sources).tolist()) == list(range(inst.k.shape[0]))
        assert sorted(np.concatenate(lay.targets).tolist()) == list(range(inst.x.shape[0]))
        assert list(lay.kb) == sorted(lay.kb) and lay.kb[0] == 0 and lay.kb[-1] == len(lay.kboxes)
        n = np.array([len(s) for s in lay.sources])
        assert n.max() < 1.5 * n.mean()                  # balanced by point count
        # the sources of rank r lie in its run of level-t_mid boxes
        for r in range(world):
            bx = sharded.box_of(inst.k[lay.sources[r]], inst.N, lay.t_mid)
            pos = {tuple(b): i for i, b in enumerate(lay.kboxes)}
            ii = np.array([pos[tuple(b)] for b in bx])
            assert ii.min() >= lay.kb[r] and ii.max() < lay.kb[r + 1]


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[3]])
def test_two_gloo_ranks_reproduce_the_unsharded_adjoint_sweep(case):
    sys.path.insert(0, HERE)
    import test_step_programs as tsp
    from paper_0801_1524_gb300 import workloads as w
    from paper_0801_1524_gb300.plan import Plan
    dim, N, p, nx, nk, seed, stages = case
    world = 2
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_adjoint, args=(r, world, port, case, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda v: v[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    inst = w.small_random(dim, N, p, nx, nk, seed, edge_fraction=0.2)
    P = Plan(inst.x, inst.k, N, p, host_only=True, stages=stages)
    L = P.info()["L"]
    opsH = np.conj(np.transpose(tsp._method_ops(p), (0, 2, 1)))
    ref = tsp.sweep(P, _stage0_tiles(P, L, 99, (p,) * dim), opsH, adjoint=True)
    col = {tuple(b): i for i, b in enumerate(P.boxes("k", L))}
    scale = np.abs(ref).max()
    seen = set()
    for rank, gL, leaves in res:
        idx = np.array([col[tuple(b)] for b in leaves])
        seen |= set(idx.tolist())
        assert np.abs(gL - ref[idx]).max() / scale < 1e-12, rank
    assert seen == set(range(len(col)))
