"""Pins for the oracle's direct sum (eq. 1.1) against results fixed by mathematics:
the inverse DFT on a lattice, the Jacobi-Anger/Bessel series for a ring of sources,
high-precision brute force, and the adjoint and transpose identities."""
import numpy as np
import pytest
from scipy.special import jv

from conftest import rel_l2
from oracle.direct import direct, direct_adjoint
from paper_0801_1524_gb300 import workloads as w


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4), (2, 5)])
def test_lattice_is_inverse_dft(dim, n):
    # x and k on the integer lattice {0..n-1}^dim with N = n: eq. 1.1 becomes
    # n^dim times numpy's inverse DFT of f laid out on the lattice.
    grid = np.stack(np.meshgrid(*[np.arange(n)] * dim, indexing="ij"), -1).reshape(-1, dim)
    f = w.gaussian_sources(grid.shape[0], seed=3)[0]
    u = direct(grid.astype(float), grid.astype(float), f, float(n))
    ref = np.fft.ifftn(f.reshape((n,) * dim)).ravel() * n ** dim
    assert rel_l2(u, ref) < 1e-12


def test_ring_of_sources_bessel_series():
    # f = 1 on n equispaced points of a circle (centre c, radius R, first angle th0):
    # u(x) = n e^{2 pi i x.c/N} sum_q i^{qn} J_{qn}(z) e^{i q n (th0 - phi_x)},
    # z = 2 pi R |x| / N, phi_x = arg x  (Jacobi-Anger expansion, sum over q in Z).
    N, R, n, th0 = 64.0, 10.0, 37, 0.3
    c = np.array([30.0, 33.0])
    th = th0 + 2 * np.pi * np.arange(n) / n
    k = c[None, :] + R * np.stack([np.cos(th), np.sin(th)], -1)
    x = w.random_points(50, N, 2, seed=11)
    u = direct(x, k, np.ones(n, complex), N)
    z = 2 * np.pi * R * np.hypot(x[:, 0], x[:, 1]) / N
    phi = np.arctan2(x[:, 1], x[:, 0])
    series = np.zeros(x.shape[0], complex)
    for q in range(-12, 13):
        m = q * n
        series += (1j ** (m % 4)) * jv(m, z) * np.exp(1j * m * (th0 - phi))
    ref = n * np.exp(2j * np.pi * (x @ c) / N) * series
    assert rel_l2(u, ref) < 1e-11


def test_bruteforce_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(5)
    N = 37.0
    x = rng.uniform(0, N, (5, 3))
    k = rng.uniform(0, N, (7, 3))
    f = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    u = direct(x, k, f, N)
    ref = []
    for xi in x:
        s = mp.mpc(0)
        for kj, fj in zip(k, f):
            dot = sum(mp.mpf(float(a)) * mp.mpf(float(b)) for a, b in zip(xi, kj))
            s += mp.expjpi(2 * dot / mp.mpf(N)) * mp.mpc(fj.real, fj.imag)
        ref.append(complex(s))
    assert rel_l2(u, np.array(ref)) < 1e-13


def test_adjoint_identity_and_transpose():
    N = 128.0
    x = w.random_points(60, N, 2, seed=1)
    k = w.random_points(45, N, 2, seed=2)
    f = w.gaussian_sources(45, seed=4)[0]
    v = w.gaussian_sources(60, seed=5)[0]
    lhs = np.vdot(v, direct(x, k, f, N))            # <A f, v>
    rhs = np.vdot(direct_adjoint(x, k, v, N), f)    # <f, A^H v>
    assert abs(lhs - rhs) / abs(lhs) < 1e-13
    # A(x, k) = A(k, x)^T: the kernel is symmetric in its two point sets.
    Axk = direct(x, k, np.eye(45), N).T
    Akx = direct(k, x, np.eye(60), N).T
    assert np.max(np.abs(Axk - Akx.T)) < 1e-12


def test_multiple_rhs_and_empty():
    N = 32.0
    x = w.random_points(20, N, 3, seed=1)
    k = w.random_points(15, N, 3, seed=2)
    f = w.gaussian_sources(15, nrhs=3, seed=4)
    u = direct(x, k, f, N)
    for r in range(3):
        assert np.allclose(u[r], direct(x, k, f[r], N), rtol=0, atol=1e-13)
    assert direct(x[:0], k, f, N).shape == (3, 0)
    assert np.all(direct(x, k[:0], np.zeros((1, 0)), N) == 0)
