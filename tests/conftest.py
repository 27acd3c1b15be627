import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: full-size cases (minutes on the host)")


def paper_eps_bands():
    """{(dim, p): (min eps_a, max eps_a)} over the paper's Tables 1-4 (tests/golden)."""
    path = os.path.join(ROOT, "tests", "golden", "paper_eps_a.txt")
    bands = {}
    with open(path) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            _tab, dim, _N, p, eps = line.split()
            key = (int(dim), int(p))
            lo, hi = bands.get(key, (float("inf"), 0.0))
            bands[key] = (min(lo, float(eps)), max(hi, float(eps)))
    return bands


def rel_l2(a, b):
    import numpy as np
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
