"""The autotuner picks the recursive step's shared-memory budget by timing candidates;
the choice changes only how work is grouped into blocks, so the result must be
bit-identical to an untuned plan, and a cached choice must be reused."""
import os

import numpy as np
import pytest

from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotuned_plan_is_identical_and_cached(tmp_path):
    from paper_0801_1524_gb300.plan import Plan
    N = 2048.0
    x = w.sample_curve(w.circle_curve(), N)
    k = w.sample_curve(w.star_curve(3), N)
    f = torch.as_tensor(w.gaussian_sources(k.shape[0], nrhs=2, seed=4), dtype=torch.complex64, device="cuda")
    cache = str(tmp_path / "tune.txt")
    tuned = Plan(x, k, N, 7, max_nrhs=2, autotune=True, tune_cache=cache)
    info = tuned.info()
    assert info["tuned_ms"] > 0 and info["smem_kb"] > 0 and info["blocks_per_sm"] >= 1
    plain = Plan(x, k, N, 7, max_nrhs=2)
    assert torch.equal(tuned.forward(f), plain.forward(f))
    assert os.path.exists(cache) and open(cache).read().strip()
    again = Plan(x, k, N, 7, max_nrhs=2, autotune=True, tune_cache=cache)
    assert again.info()["tuned_ms"] == 0                 # taken from the cache
    assert again.info()["smem_kb"] == info["smem_kb"]
