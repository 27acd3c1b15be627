"""Seeded synthetic workloads: point sets on curves and surfaces, and source vectors.

This module is shared by the CUDA path, the oracle tests and the benchmark. It only
draws and places points; it holds none of the transform's arithmetic.

The paper samples its curves at a fixed number of points per unit length (Sec. 3.1)
and its surfaces at a fixed number of points per unit area (Sec. 3.2), with random
mean-zero sources.  The shapes here (circles, a perturbed ellipse, random star-shaped
curves, a sphere) stand in for the paper's ellipses, "smooth curves", F16 and
submarine meshes, which are only shown in figures.

Every point set lies in [0, N]^d (the unit box scaled by N, eq. 1.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------------------
# curves in the unit square


def circle_curve(radius: float = 0.4, centre=(0.5, 0.5)):
    cx, cy = centre

    def curve(theta):
        return np.stack([cx + radius * np.cos(theta), cy + radius * np.sin(theta)], axis=-1)

    return curve


def perturbed_ellipse_curve(a: float = 0.45, b: float = 0.3, eps: float = 0.03, m: int = 5,
                            centre=(0.5, 0.5)):
    """(0.5,0.5) + (a cos t, b sin t) + eps sin(m t) (cos t, sin t)."""
    cx, cy = centre

    def curve(theta):
        pert = eps * np.sin(m * theta)
        return np.stack([cx + a * np.cos(theta) + pert * np.cos(theta),
                         cy + b * np.sin(theta) + pert * np.sin(theta)], axis=-1)

    return curve


def star_curve(seed: int, base: float = 0.35, modes: int = 6, amp: float = 0.02,
               centre=(0.5, 0.5)):
    """r(t) = base + sum_{m=1..modes} a_m cos(m t + phi_m), a_m ~ U(0, amp/m), phi_m ~ U(0, 2 pi).

    The amplitudes are drawn first, then the phases, from numpy default_rng(seed).
    """
    rng = np.random.default_rng(seed)
    mm = np.arange(1, modes + 1)
    a_m = rng.uniform(0.0, amp / mm)
    phi_m = rng.uniform(0.0, 2.0 * np.pi, size=modes)
    cx, cy = centre

    def curve(theta):
        th = np.asarray(theta)
        r = base + np.sum(a_m[:, None] * np.cos(mm[:, None] * th.reshape(1, -1) + phi_m[:, None]),
                          axis=0).reshape(th.shape)
        return np.stack([cx + r * np.cos(th), cy + r * np.sin(th)], axis=-1)

    return curve


def sample_curve(curve, N: float, per_unit_length: float = 4.0, table: int = 200_000):
    """Samples the closed curve N*curve uniformly in arclength, starting at theta = 0.

    n = round(per_unit_length * length(N*curve)); the length and theta(s) come from a
    dense polyline of `table` segments, inverted by linear interpolation.
    """
    th = np.linspace(0.0, 2.0 * np.pi, table + 1)
    pts = curve(th) * float(N)
    seg = np.hypot(np.diff(pts[:, 0]), np.diff(pts[:, 1]))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    length = s[-1]
    n = int(round(per_unit_length * length))
    si = np.arange(n) * (length / n)
    th_i = np.interp(si, s, th)
    out = curve(th_i) * float(N)
    return np.clip(out, 0.0, float(N))


def fibonacci_sphere(N: float, radius: float = 0.4, centre=(0.5, 0.5, 0.5),
                     per_unit_area: float = 1.0):
    """Fibonacci lattice on the sphere N*(centre + radius*S^2), n = round(area * density)."""
    R = radius * float(N)
    n = int(round(4.0 * np.pi * R * R * per_unit_area))
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - 2.0 * (i + 0.5) / n
    phi = i * np.pi * (3.0 - np.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    c = np.asarray(centre, dtype=np.float64)
    pts = float(N) * c[None, :] + R * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=-1)
    return np.clip(pts, 0.0, float(N))


def gaussian_sources(n: int, nrhs: int = 1, seed: int = 0, dtype=np.complex128):
    """f with i.i.d. N(0,1) real and imaginary parts: default_rng(seed).standard_normal((nrhs, n, 2))."""
    a = np.random.default_rng(seed).standard_normal((nrhs, n, 2))
    f = a[..., 0] + 1j * a[..., 1]
    return f.astype(dtype)


def random_points(n: int, N: float, dim: int, seed: int, edge_fraction: float = 0.0):
    """Uniform points in [0,N]^dim; a fraction is snapped to the grid of spacing
    h = sqrt(N / 2^ceil(log2 N)) (the unit grid when N is a power of two) and to N itself."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, float(N), size=(n, dim))
    if edge_fraction > 0 and n > 0:
        m = max(1, int(edge_fraction * n))
        idx = rng.choice(n, size=min(m, n), replace=False)
        Np = 2.0 ** max(0, math.ceil(math.log2(float(N)) - 1e-12)) if N > 1 else 1.0
        h = math.sqrt(float(N) / Np)
        pts[idx] = np.floor(pts[idx] / h) * h
        if len(idx) > 1:
            pts[idx[0], :] = float(N)
            pts[idx[1], 0] = float(N)
    return pts


# ----------------------------------------------------------------------------------------
# named workloads


@dataclass
class Instance:
    name: str
    dim: int
    N: float
    p: int
    x: np.ndarray            # targets  [nx, dim] float64 in [0,N]^dim
    k: np.ndarray            # sources  [nk, dim] float64 in [0,N]^dim
    nrhs: int = 1
    f_seed: int = 0
    meta: dict = field(default_factory=dict)

    def sources(self, dtype=np.complex128, nrhs: int | None = None, seed: int | None = None):
        return gaussian_sources(self.k.shape[0], self.nrhs if nrhs is None else nrhs,
                                self.f_seed if seed is None else seed, dtype)


def circle256() -> Instance:
    """2D, N=256: X = K = circle r=0.4 about (0.5,0.5), 4 points per unit length, p=5."""
    N = 256.0
    pts = sample_curve(circle_curve(), N)
    return Instance("circle256_p5", 2, N, 5, pts, pts.copy())


def curve8192(p: int = 7) -> Instance:
    """2D, N=8192: X = circle r=0.4; K = ellipse (0.45,0.3) + 0.03 sin(5 theta) radial; p=7."""
    N = 8192.0
    return Instance(f"curve8192_p{p}", 2, N, p, sample_curve(circle_curve(), N),
                    sample_curve(perturbed_ellipse_curve(), N))


def sphere128(p: int = 5) -> Instance:
    """3D, N=128: X = K = Fibonacci sphere r=0.4, 1 point per unit area, p=5."""
    N = 128.0
    pts = fibonacci_sphere(N)
    return Instance(f"sphere128_p{p}", 3, N, p, pts, pts.copy())


def star32768(p: int = 7) -> Instance:
    """2D, N=32768: X = circle r=0.4; K = star-shaped curve with seed 7; p=7."""
    N = 32768.0
    return Instance(f"star32768_p{p}", 2, N, p, sample_curve(circle_curve(), N),
                    sample_curve(star_curve(7), N))


def batch_sizes(count: int = 64, lo: float = 512.0, hi: float = 16384.0, seed: int = 0):
    """N_i log-uniform in [lo, hi] from default_rng(seed) (real-valued, as drawn), and the
    nearest powers of two (a comparison setting with unit leaves only)."""
    rng = np.random.default_rng(seed)
    n_exact = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    n_pow2 = 2.0 ** np.round(np.log2(n_exact))
    return n_exact, n_pow2


def star_batch(count: int = 64, p: int = 7, nrhs: int = 16, power_of_two: bool = False,
               seed: int = 0) -> list[Instance]:
    """64 instances of star-shaped curve pairs of the drawn N (power_of_two: rounded to the
    nearest power of two); instance i uses X seed 2i+1000, K seed 2i+1001."""
    n_exact, n_pow2 = batch_sizes(count, seed=seed)
    out = []
    for i in range(count):
        N = float(n_pow2[i] if power_of_two else n_exact[i])
        x = sample_curve(star_curve(2 * i + 1000), N)
        k = sample_curve(star_curve(2 * i + 1001), N)
        out.append(Instance(f"star_batch{i}", 2, N, p, x, k, nrhs=nrhs, f_seed=i,
                            meta={"N_drawn": float(n_exact[i])}))
    return out


def small_random(dim: int, N: float, p: int, nx: int, nk: int, seed: int,
                 edge_fraction: float = 0.1) -> Instance:
    """Uniform random points (not on a curve), with some on box edges and at N."""
    x = random_points(nx, N, dim, seed, edge_fraction)
    k = random_points(nk, N, dim, seed + 1, edge_fraction)
    return Instance(f"random{dim}d_N{int(N)}_p{p}", dim, float(N), p, x, k, f_seed=seed + 2)


WORKLOADS = {
    "circle256": circle256,
    "curve8192": curve8192,
    "sphere128": sphere128,
    "star32768": star32768,
}
