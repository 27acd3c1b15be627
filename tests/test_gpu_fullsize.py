"""Parity at the full workload sizes, in the launch configuration the benchmark times.

  curve8192 (2D, N=8192, p=7)   FP32 and FP64 paths against the oracle's butterfly
                                (1e-6 / 1e-9) and, on 4096 sampled targets, against the
                                direct sum within the paper's eps_a band (Tables 1-2).
  sphere128 (3D, N=128, p=5)    FP32 and FP64 paths against the oracle's butterfly
                                (1e-6 / 1e-9), sampled direct sum within the 3D band.
  star32768 (2D, N=32768, p=7)  forward and adjoint on sampled outputs against the direct
                                sums (band), FP32 against FP64 (1e-6), the adjoint's
                                transpose identity, and the gradient of
                                L(f) = ||B f - u_obs||^2 against central differences.
"""
import numpy as np
import pytest

import oracle.butterfly as ob
from conftest import paper_eps_bands, rel_l2
from oracle.direct import direct, direct_adjoint
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]
BANDS = paper_eps_bands()


def _plan(inst, prec, nrhs=1):
    from paper_0801_1524_gb300.plan import Plan
    return Plan(inst.x, inst.k, inst.N, inst.p, precision=prec, max_nrhs=nrhs)


def _run(plan, f, dtype):
    u = plan.forward(torch.as_tensor(f, dtype=dtype, device="cuda"))
    return u.cpu().numpy().astype(np.complex128)


def _sample(n, m=4096, seed=12345):
    return np.random.default_rng(seed).choice(n, size=min(n, m), replace=False)


def test_curve8192_against_oracle_butterfly():
    inst = w.curve8192()
    f = inst.sources()[0]
    ref = ob.butterfly(inst.x, inst.k, f, inst.N, inst.p)
    u32 = _run(_plan(inst, "fp32"), f, torch.complex64)
    u64 = _run(_plan(inst, "fp64"), f, torch.complex128)
    assert rel_l2(u64, ref) < 1e-9
    assert rel_l2(u32, ref) < 1e-6
    S = _sample(inst.x.shape[0])
    exact = direct(inst.x[S], inst.k, f, inst.N)
    assert rel_l2(u64[S], exact) < 2 * BANDS[(2, inst.p)][1]


def test_sphere128_against_oracle_butterfly():
    inst = w.sphere128()
    f = inst.sources()[0]
    ref = ob.butterfly(inst.x, inst.k, f, inst.N, inst.p)
    u32 = _run(_plan(inst, "fp32"), f, torch.complex64)
    u64 = _run(_plan(inst, "fp64"), f, torch.complex128)
    assert rel_l2(u64, ref) < 1e-9
    assert rel_l2(u32, ref) < 1e-6
    S = _sample(inst.x.shape[0])
    exact = direct(inst.x[S], inst.k, f, inst.N)
    assert rel_l2(u64[S], exact) < 2 * BANDS[(3, inst.p)][1]


def test_star32768_forward_adjoint_and_gradient():
    from paper_0801_1524_gb300.plan import butterfly
    inst = w.star32768()
    nx, nk = inst.x.shape[0], inst.k.shape[0]
    P32, P64 = _plan(inst, "fp32"), _plan(inst, "fp64")
    f = inst.sources()[0]
    u32 = _run(P32, f, torch.complex64)
    u64 = _run(P64, f, torch.complex128)
    assert rel_l2(u32, u64) < 1e-6
    S = _sample(nx)
    assert rel_l2(u64[S], direct(inst.x[S], inst.k, f, inst.N)) < 2 * BANDS[(2, 7)][1]
    # adjoint: transpose identity and sampled direct adjoint sum
    v = w.gaussian_sources(nx, seed=3)[0]
    vt = torch.as_tensor(v, device="cuda")
    g64 = P64.adjoint(vt).cpu().numpy()
    g32 = P32.adjoint(vt.to(torch.complex64)).cpu().numpy().astype(np.complex128)
    assert rel_l2(g32, g64) < 1e-6
    lhs, rhs = np.vdot(v, u64), np.vdot(g64, f)
    assert abs(lhs - rhs) / (np.linalg.norm(u64) * np.linalg.norm(v)) < 1e-12
    Sk = _sample(nk)
    assert rel_l2(g64[Sk], direct_adjoint(inst.x, inst.k[Sk], v, inst.N)) < 2 * BANDS[(2, 7)][1]
    # gradient of L(f) = ||B f - u_obs||^2, u_obs from f* (seed 8) through the FP64 path
    fstar = torch.as_tensor(inst.sources(seed=8)[0], device="cuda")
    u_obs = P64.forward(fstar)
    f0 = torch.as_tensor(f, device="cuda")
    x32 = f0.to(torch.complex64).requires_grad_(True)
    (butterfly(x32, P32).to(torch.complex128) - u_obs).abs().pow(2).sum().backward()
    g_ref = 2.0 * P64.adjoint(P64.forward(f0) - u_obs)
    assert rel_l2(x32.grad.to(torch.complex128).cpu().numpy(), g_ref.cpu().numpy()) < 1e-5
    rng = np.random.default_rng(7)
    h = 1e-3
    fd, an = [], []
    for j in rng.choice(nk, 32, replace=False):
        for unit in (1.0, 1j):
            e = torch.zeros_like(f0)
            e[j] = unit * h
            lp = (P64.forward(f0 + e) - u_obs).abs().pow(2).sum().item()
            lm = (P64.forward(f0 - e) - u_obs).abs().pow(2).sum().item()
            fd.append((lp - lm) / (2 * h))
            an.append(g_ref[j].real.item() if unit == 1.0 else g_ref[j].imag.item())
    assert rel_l2(np.array(an), np.array(fd)) < 1e-6
