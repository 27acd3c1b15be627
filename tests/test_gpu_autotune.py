"""The autotuner picks the recursive step's configuration by timing candidates: the
shared-memory budget per block (how many box pairs a block takes at a time, how many
blocks share an SM), the stages per launch in 2D, and, for FP32 plans with at least eight
right-hand sides, the tensor-core step.  The choice only changes how the same sweep is
grouped and issued, so a tuned plan equals an untuned plan built with the chosen
configuration bit for bit, and stays within the FP32 gate of the default plan; a cached
choice is reused; a batch of plans built with the tuned configuration equals the same
batch built by hand."""
import os

import numpy as np
import pytest

from conftest import rel_l2
from paper_0801_1524_gb300 import native
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {native.BFLY_PREC_FP32: "fp32", native.BFLY_PREC_TC: "tc", native.BFLY_PREC_FP64: "fp64"}


def _chosen(plan):
    i = plan.info()
    prec = "fp32g" if i["rhs_groups"] else PREC[i["prec"]]
    return dict(smem_kb=i["smem_kb"], stages=i["stages_per_launch"], precision=prec, dataflow=bool(i["dataflow"]))


@pytest.mark.parametrize("nrhs", [2, 16])
def test_autotuned_plan_is_identical_and_cached(tmp_path, nrhs):
    from paper_0801_1524_gb300.plan import Plan
    N = 2048.0
    x = w.sample_curve(w.circle_curve(), N)
    k = w.sample_curve(w.star_curve(3), N)
    f = torch.as_tensor(w.gaussian_sources(k.shape[0], nrhs=nrhs, seed=4), dtype=torch.complex64, device="cuda")
    cache = str(tmp_path / "tune.txt")
    tuned = Plan(x, k, N, 7, max_nrhs=nrhs, autotune=True, tune_cache=cache)
    info = tuned.info()
    assert info["tuned_ms"] > 0 and info["smem_kb"] > 0 and info["blocks_per_sm"] >= 1
    assert info["stages_per_launch"] in (1, 2, 3)
    if nrhs < 8:
        assert info["prec"] == native.BFLY_PREC_FP32   # the tensor-core step needs 8 columns
    ch = _chosen(tuned)
    by_hand = Plan(x, k, N, 7, max_nrhs=nrhs, **ch)
    assert by_hand.info()["smem_kb"] == ch["smem_kb"]
    u = tuned.forward(f)
    assert torch.equal(u, by_hand.forward(f))
    plain = Plan(x, k, N, 7, max_nrhs=nrhs)
    ref = plain.forward(f).cpu().numpy().astype(np.complex128)
    got = u.cpu().numpy().astype(np.complex128)
    for r in range(nrhs):
        assert rel_l2(got[r], ref[r]) < 2e-6
    assert os.path.exists(cache) and open(cache).read().strip()
    again = Plan(x, k, N, 7, max_nrhs=nrhs, autotune=True, tune_cache=cache)
    assert again.info()["tuned_ms"] == 0                 # taken from the cache
    assert _chosen(again) == ch


def test_tuned_batch_equals_the_same_batch_by_hand(tmp_path):
    # the batched workload's way of tuning: the largest instance is tuned, its configuration
    # is used for every plan of the batch
    from paper_0801_1524_gb300.plan import Batch, Plan
    sizes = (300.5, 1000.0, 2500.0, 700.0)
    insts = [w.Instance(f"b{i}", 2, N, 7, w.sample_curve(w.star_curve(2 * i + 1000), N),
                        w.sample_curve(w.star_curve(2 * i + 1001), N), nrhs=8, f_seed=i)
             for i, N in enumerate(sizes)]
    big = max(insts, key=lambda I: I.N)
    ch = _chosen(Plan(big.x, big.k, big.N, 7, max_nrhs=8, autotune=True, tune_cache=str(tmp_path / "t.txt")))
    fs = [torch.as_tensor(I.sources(), dtype=torch.complex64, device="cuda") for I in insts]
    outs = []
    for _ in range(2):
        plans = [Plan(I.x, I.k, I.N, 7, max_nrhs=8, **ch) for I in insts]
        b = Batch(plans)
        outs.append(b.forward(fs))
        torch.cuda.synchronize()
        assert b.device_status() == 0
    for a, c in zip(*outs):
        assert torch.equal(a, c)
    ref = [Plan(I.x, I.k, I.N, 7, max_nrhs=8).forward(f) for I, f in zip(insts, fs)]
    for a, r in zip(outs[0], ref):
        for j in range(8):
            assert rel_l2(a[j].cpu().numpy(), r[j].cpu().numpy()) < 2e-6
