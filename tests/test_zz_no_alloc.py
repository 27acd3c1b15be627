"""bfly_execute_noalloc, the entry point for callers that cannot allocate device memory
when they run the transform (their device memory belongs to an external allocator or a
fixed budget, or cudaMalloc's device synchronisation is not acceptable on their execution
path): the same forward sweep as bfly_execute with the charge buffers taken from the
library's static device workspace.  Its output must match bfly_execute's on two calls in
a row (the workspace keeps the previous call's contents), also with several right-hand
sides, and requests larger than the workspace must be refused with a clear error.  This
file is collected last."""
import ctypes

import numpy as np
import pytest

from conftest import rel_l2
from paper_0801_1524_gb300 import native
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call_noalloc(plan, f, u):
    lib = native.load()
    dtype = native.BFLY_C128 if f.dtype == torch.complex128 else native.BFLY_C64
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.bfly_execute_noalloc(plan._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                    1 if f.dim() == 1 else f.shape[0], dtype, stream)


@pytest.mark.parametrize("prec,dtype,tol", [("fp32", torch.complex64, 1e-6), ("fp64", torch.complex128, 1e-9),
                                            ("tc", torch.complex64, 1e-6)])
def test_noalloc_matches_execute_on_two_calls(prec, dtype, tol):
    from paper_0801_1524_gb300.plan import Plan
    N, p = 1024.0, 7
    x = w.sample_curve(w.circle_curve(), N)
    k = w.sample_curve(w.perturbed_ellipse_curve(), N)
    plan = Plan(x, k, N, p, precision=prec)
    f1 = torch.as_tensor(w.gaussian_sources(k.shape[0], seed=1)[0], dtype=dtype, device="cuda")
    f2 = torch.as_tensor(w.gaussian_sources(k.shape[0], seed=2)[0], dtype=dtype, device="cuda")
    for f in (f1, f2):  # two calls in a row on the shared workspace
        ref = plan.forward(f)
        u = torch.empty_like(ref)
        assert _call_noalloc(plan, f, u) == native.BFLY_OK, native.load().bfly_last_error()
        torch.cuda.synchronize()
        assert rel_l2(u.cpu().numpy(), ref.cpu().numpy()) <= tol


def test_noalloc_refuses_a_plan_beyond_the_workspace():
    from paper_0801_1524_gb300.plan import Plan
    inst = w.curve8192()  # largest stage ~89k tiles of 49 complex128: beyond 32 MiB
    plan = Plan(inst.x, inst.k, inst.N, inst.p, precision="fp64")
    f = torch.zeros(inst.k.shape[0], dtype=torch.complex128, device="cuda")
    u = torch.zeros(inst.x.shape[0], dtype=torch.complex128, device="cuda")
    assert _call_noalloc(plan, f, u) == native.BFLY_ERR_INVALID_ARG
    assert "static workspace" in native.load().bfly_last_error().decode()


def test_noalloc_several_rhs_and_the_size_limit():
    # N = 2048, p = 7, FP32: the largest stage holds 22,232 tiles of 50 complex64 values
    # (8.9 MB per right-hand side), so three right-hand sides fit the 32 MiB buffer and
    # four do not
    from paper_0801_1524_gb300.plan import Plan
    N = 2048.0
    x = w.sample_curve(w.circle_curve(), N)
    k = w.sample_curve(w.perturbed_ellipse_curve(), N)
    plan = Plan(x, k, N, 7, precision="fp32", max_nrhs=4)
    per_rhs = plan.info()["max_pairs"] * 50 * 8
    fit = (32 << 20) // per_rhs
    assert fit == 3
    for seed in (5, 6):  # two calls in a row
        f = torch.as_tensor(w.gaussian_sources(k.shape[0], nrhs=fit, seed=seed), dtype=torch.complex64,
                            device="cuda")
        ref = plan.forward(f)
        u = torch.empty_like(ref)
        assert _call_noalloc(plan, f, u) == native.BFLY_OK, native.load().bfly_last_error()
        torch.cuda.synchronize()
        for r in range(fit):
            assert rel_l2(u[r].cpu().numpy(), ref[r].cpu().numpy()) <= 1e-6
    f4 = torch.zeros((fit + 1, k.shape[0]), dtype=torch.complex64, device="cuda")
    u4 = torch.zeros((fit + 1, x.shape[0]), dtype=torch.complex64, device="cuda")
    assert _call_noalloc(plan, f4, u4) == native.BFLY_ERR_INVALID_ARG
    assert "static workspace" in native.load().bfly_last_error().decode()
