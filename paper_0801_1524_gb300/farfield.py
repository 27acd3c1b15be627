"""Far-field pattern of a surface density through the butterfly (eq. 1.2 of Sec. 1).

The far field of a density f on a surface Gamma in the unit cube, at frequency N, is

    u_inf(xh) = int_Gamma exp(-i N xh . y) f(y) ds(y),     xh on the unit sphere.

With a quadrature y_j, w_j of Gamma this is a sum of the form of eq. 1.1.  Put the sources
at k_j = M y_j in [0, M]^3 and the targets at x_i = (M / 2) (1 - xh_i) in [0, M]^3 with
M = N / pi; then 2 pi x_i . k_j / M = N sum_d y_jd - N xh_i . y_j, so

    u_inf(xh_i) = sum_j exp(2 pi i x_i . k_j / M) g_j,    g_j = w_j f_j exp(-i N sum_d y_jd),

the transform of eq. 1.1 with domain size M (not a power of two: the plan scales the
points, see bfly_plan_create).  The strengths g_j are prepared on the host in FP64 (a
unimodular factor per source); the transform runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from .plan import Plan


def directions_fibonacci(n: int) -> np.ndarray:
    """n directions on the unit sphere (Fibonacci lattice), [n, 3]."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - 2.0 * (i + 0.5) / n
    phi = i * np.pi * (3.0 - np.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=-1)


def sphere_quadrature(n: int, radius: float = 0.4, centre=(0.5, 0.5, 0.5)):
    """Equal-weight quadrature of the sphere |y - centre| = radius on n Fibonacci points:
    returns y [n, 3] and w [n] (each the area / n)."""
    y = np.asarray(centre, dtype=np.float64)[None, :] + radius * directions_fibonacci(n)
    return y, np.full(n, 4.0 * np.pi * radius * radius / n)


def mapped_problem(y, w, f, N: float, xh):
    """The far-field sum as eq. 1.1: (x [nx, 3], k [nk, 3], g [nrhs, nk], M)."""
    y = np.asarray(y, dtype=np.float64)
    xh = np.asarray(xh, dtype=np.float64)
    if y.min() < 0.0 or y.max() > 1.0:
        raise ValueError("the surface must lie in the unit cube")
    M = float(N) / np.pi
    k = np.clip(M * y, 0.0, M)
    x = np.clip(0.5 * M * (1.0 - xh), 0.0, M)
    g = np.atleast_2d(np.asarray(f, dtype=np.complex128)) * (w * np.exp(-1j * float(N) * y.sum(axis=1)))[None, :]
    return x, k, g, M


class FarField:
    """u_inf at the directions xh for densities on the quadrature nodes y (weights w) at
    frequency N: a butterfly plan of the mapped problem (3D, p charges per axis)."""

    def __init__(self, y, w, xh, N: float, p: int = 5, precision: str = "fp32", max_nrhs: int = 1):
        self.y = np.asarray(y, dtype=np.float64)
        self.w = np.asarray(w, dtype=np.float64)
        self.xh = np.asarray(xh, dtype=np.float64)
        self.N = float(N)
        x, k, _, self.M = mapped_problem(self.y, self.w, np.ones(self.y.shape[0]), self.N, self.xh)
        self.plan = Plan(x, k, self.M, p, precision=precision, max_nrhs=max_nrhs)
        self._phase = self.w * np.exp(-1j * self.N * self.y.sum(axis=1))

    def strengths(self, f):
        """g_j = w_j f_j exp(-i N sum_d y_jd) for densities f [nk] or [nrhs, nk]."""
        return np.atleast_2d(np.asarray(f, dtype=np.complex128)) * self._phase[None, :]

    def __call__(self, f, dtype=None):
        """u_inf [nrhs, n_directions] (a torch tensor on the plan's device)."""
        import torch
        dt = dtype or (torch.complex128 if self.plan.precision == "fp64" else torch.complex64)
        g = torch.as_tensor(self.strengths(f)).to(device="cuda", dtype=dt)
        return self.plan.forward(g)

