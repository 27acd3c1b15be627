"""CPU pins of the far-field mapping (eq. 1.2 onto eq. 1.1; paper_0801_1524_gb300.farfield):
the oracle's direct sum of the mapped problem equals the far-field sum by its definition,
and the quadrature of the sphere reproduces the closed form of a uniform density."""
import numpy as np

from oracle.direct import direct
from paper_0801_1524_gb300 import farfield as ff


def _definition(xh, y, w, f, N):
    return np.exp(-1j * N * (xh @ y.T)) @ (w * f)


def test_mapped_sum_equals_the_far_field_sum():
    N = 24.0
    y, w = ff.sphere_quadrature(3000)
    xh = ff.directions_fibonacci(300)
    f = np.random.default_rng(1).standard_normal(3000) + 0j
    x, k, g, M = ff.mapped_problem(y, w, f, N, xh)
    assert abs(M - N / np.pi) < 1e-15 and x.min() >= 0 and x.max() <= M and k.max() <= M
    a = direct(x, k, g[0], M)
    b = _definition(xh, y, w, f, N)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12


def test_sphere_quadrature_matches_the_closed_form():
    # f = 1 on the sphere |y - c| = R: u_inf = 4 pi R^2 sin(NR)/(NR) exp(-i N xh . c)
    N, R, c = 16.0, 0.4, np.array([0.5, 0.5, 0.5])
    y, w = ff.sphere_quadrature(20000)
    xh = ff.directions_fibonacci(200)
    exact = 4 * np.pi * R * R * np.sin(N * R) / (N * R) * np.exp(-1j * N * (xh @ c))
    got = _definition(xh, y, w, np.ones(20000), N)
    assert np.linalg.norm(got - exact) / np.linalg.norm(exact) < 1e-4
    assert abs(w.sum() - 4 * np.pi * R * R) < 1e-12
