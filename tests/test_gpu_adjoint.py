"""The adjoint sweep (the exact conjugate transpose of the forward butterfly) and the
autograd function built on it."""
import numpy as np
import pytest

import oracle.butterfly as ob
from conftest import paper_eps_bands, rel_l2
from oracle.direct import direct_adjoint
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
BANDS = paper_eps_bands()


def _plan(inst, prec, nrhs=1):
    from paper_0801_1524_gb300.plan import Plan
    return Plan(inst.x, inst.k, inst.N, inst.p, precision=prec, max_nrhs=nrhs)


def _gpu(a, dtype=torch.complex128):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("dim,N,p", [(2, 64.0, 5), (2, 256.0, 7), (3, 8.0, 5), (2, 1.0, 3), (2, 300.0, 7),
                                     (3, 10.0, 5)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dot_product_identity(dim, N, p, prec):
    inst = w.small_random(dim, N, p, 700, 600, 21)
    P = _plan(inst, prec)
    f = _gpu(inst.sources()[0])
    v = _gpu(w.gaussian_sources(inst.x.shape[0], seed=22)[0])
    lhs = torch.vdot(v, P.forward(f)).item()
    rhs = torch.vdot(P.adjoint(v), f).item()
    scale = (torch.linalg.norm(P.forward(f)) * torch.linalg.norm(v)).item()
    assert abs(lhs - rhs) / scale < (1e-13 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("dim,N,p", [(2, 16.0, 5), (3, 4.0, 3), (2, 20.0, 5), (3, 6.0, 3)])
def test_adjoint_equals_transpose_of_oracle_matrix(dim, N, p):
    inst = w.small_random(dim, N, p, 60, 50, 23)
    B = ob.butterfly_matrix(inst.x, inst.k, N, p)       # [nx, nk] from the oracle
    v = w.gaussian_sources(inst.x.shape[0], seed=24)[0]
    ref = B.conj().T @ v
    got = _plan(inst, "fp64").adjoint(_gpu(v)).cpu().numpy()
    assert rel_l2(got, ref) < 1e-9


def test_adjoint_against_direct_adjoint_sum():
    N, p = 512.0, 7
    x = w.sample_curve(w.circle_curve(), N)
    k = w.sample_curve(w.star_curve(7), N)
    inst = w.Instance("adj", 2, N, p, x, k)
    v = w.gaussian_sources(x.shape[0], nrhs=2, seed=25)
    got = _plan(inst, "fp32", nrhs=2).adjoint(_gpu(v, torch.complex64)).cpu().numpy()
    ref = direct_adjoint(x, k, v, N)
    assert rel_l2(got, ref) < 2 * BANDS[(2, p)][1]


def test_autograd_gradient_and_finite_differences():
    from paper_0801_1524_gb300.plan import butterfly
    N, p = 256.0, 7
    x = w.sample_curve(w.circle_curve(), N)
    k = w.sample_curve(w.star_curve(7), N)
    inst = w.Instance("grad", 2, N, p, x, k)
    P64 = _plan(inst, "fp64")
    P32 = _plan(inst, "fp32")
    fstar = _gpu(inst.sources(seed=8)[0])
    u_obs = P64.forward(fstar)
    f0 = _gpu(inst.sources(seed=3)[0])

    def loss(plan, f):
        r = plan.forward(f) - u_obs
        return (r.abs() ** 2).sum()

    f = f0.clone().to(torch.complex64).requires_grad_(True)
    L = (butterfly(f, P32).to(torch.complex128) - u_obs).abs().pow(2).sum()
    L.backward()
    g32 = f.grad.to(torch.complex128)
    f64 = f0.clone().requires_grad_(True)
    L64 = (butterfly(f64, P64) - u_obs).abs().pow(2).sum()
    L64.backward()
    g64 = f64.grad
    # closed form of PyTorch's convention: dL/dRe f + i dL/dIm f = 2 B^H (B f - u_obs)
    g_ref = 2.0 * P64.adjoint(P64.forward(f0) - u_obs)
    assert rel_l2(g64.cpu().numpy(), g_ref.cpu().numpy()) < 1e-12
    assert rel_l2(g32.cpu().numpy(), g_ref.cpu().numpy()) < 1e-5
    # central differences with step h on 32 random entries, real and imaginary parts
    rng = np.random.default_rng(7)
    idx = rng.choice(k.shape[0], 32, replace=False)
    h = 1e-3
    fd, an = [], []
    for j in idx:
        for unit in (1.0, 1j):
            e = torch.zeros_like(f0)
            e[j] = unit * h
            d = (loss(P64, f0 + e) - loss(P64, f0 - e)).item() / (2 * h)
            fd.append(d)
            an.append(g64[j].real.item() if unit == 1.0 else g64[j].imag.item())
    assert rel_l2(np.array(an), np.array(fd)) < 1e-8
