"""Far-field pattern (eq. 1.2, Sec. 1) through the butterfly: the far field of a density on
the synthetic sphere (the stand-in for the paper's scatterer surfaces) at frequency N,
mapped onto eq. 1.1 (paper_0801_1524_gb300.farfield).  Checked against

* the far-field sum by its definition, sum_j w_j f_j exp(-i N xh_i . y_j) (numpy, FP64),
  within the 3D band of the paper's Tables 3-4 for the plan's p;
* the oracle's direct sum (eq. 1.1) of the mapped problem (same band), which pins the
  mapping x = (M/2)(1 - xh), k = M y, M = N / pi;
* for f = 1, the closed form 4 pi R^2 j0(N R) exp(-i N xh . c) of a uniform density on
  the sphere of radius R and centre c, within the quadrature error of the Fibonacci nodes
  (about 1e-4 relative at 20,000 nodes and N = 32) plus the band.
"""
import numpy as np
import pytest

from conftest import paper_eps_bands, rel_l2
from oracle.direct import direct

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
BANDS = paper_eps_bands()


def _exact_uniform_sphere(xh, N, radius=0.4, centre=(0.5, 0.5, 0.5)):
    z = N * radius
    return 4.0 * np.pi * radius ** 2 * (np.sin(z) / z) * np.exp(-1j * N * (xh @ np.asarray(centre)))


def _definition(xh, y, w, f, N):
    out = np.zeros(xh.shape[0], dtype=np.complex128)
    for a in range(0, xh.shape[0], 512):
        out[a:a + 512] = np.exp(-1j * N * (xh[a:a + 512] @ y.T)) @ (w * f)
    return out


@pytest.mark.parametrize("prec,p", [("fp64", 5), ("fp32", 5), ("fp64", 7)])
def test_far_field_of_the_sphere(prec, p):
    from paper_0801_1524_gb300 import farfield as ff
    N = 32.0
    y, w = ff.sphere_quadrature(20000)
    xh = ff.directions_fibonacci(3000)
    F = ff.FarField(y, w, xh, N, p=p, precision=prec, max_nrhs=2)
    rng = np.random.default_rng(5)
    f = np.stack([np.ones(y.shape[0], dtype=np.complex128),
                  rng.standard_normal(y.shape[0]) + 1j * rng.standard_normal(y.shape[0])])
    u = F(f).cpu().numpy().astype(np.complex128)
    torch.cuda.synchronize()
    band = 2 * BANDS[(3, p)][1]
    # against the definition of the far field and the oracle's sum of the mapped problem
    for r in range(2):
        ref = _definition(xh, y, w, f[r], N)
        assert rel_l2(u[r], ref) < band
    x, k, g, M = ff.mapped_problem(y, w, f[1], N, xh)
    S = np.random.default_rng(6).choice(xh.shape[0], 400, replace=False)
    assert rel_l2(u[1][S], direct(x[S], k, g[0], M)) < band
    # a uniform density: the closed form, up to the quadrature error
    assert rel_l2(u[0], _exact_uniform_sphere(xh, N)) < 3e-4 + band
