"""The multi-rank path of the benchmark on CPU: two gloo ranks (one process each, as
torchrun starts them) agree on the job's step time (the maximum over ranks) and the
whole-job throughput counts the transforms of every rank.  The transform itself does not
shard (independent replicas); no collective is on its data path."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(times[rank], dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, bench.replica_value(world, ms)))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    times = [0.5, 0.8]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(ms == 0.8 for _, ms, _ in res)
    assert all(abs(v - 2 * 1e3 / 0.8) < 1e-9 for _, _, v in res)


def test_single_rank_is_unchanged():
    import importlib
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    assert bench.max_over_ranks(1.25, None) == 1.25
    assert bench.replica_value(1, 2.0) == 500.0
