"""Parity of the CUDA butterfly (through the C ABI) with the oracle.

Tolerances (relative L2 over all outputs):
  FP64 path vs the oracle's butterfly          1e-9   (the target for the FP64 path)
  FP32 path vs the oracle's butterfly, p <= 7  1e-6   (the target for the FP32 path)
  FP32 path, p = 9                             4e-6   (FP32 rounding through the sweep grows
                                                       with the operator norm; see the
                                                       precision notes of the design)
  every path vs the direct sum (eq. 1.1)       2x the paper's largest eps_a for (dim, p)
"""
import numpy as np
import pytest

import oracle.butterfly as ob
from conftest import paper_eps_bands, rel_l2
from oracle.direct import direct, direct_adjoint
from paper_0801_1524_gb300 import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BANDS = paper_eps_bands()
TOL64 = 1e-9


def tol32(p):
    return 1e-6 if p <= 7 else 4e-6


def _plan(inst, prec, nrhs=1):
    from paper_0801_1524_gb300.plan import Plan
    return Plan(inst.x, inst.k, inst.N, inst.p, precision=prec, max_nrhs=nrhs)


def _gpu(a, dtype=torch.complex128):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _fwd(inst, f, prec, dtype=torch.complex128):
    P = _plan(inst, prec, nrhs=1 if f.ndim == 1 else f.shape[0])
    u = P.forward(_gpu(f, dtype))
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.complex128)


SMALL = [
    # (dim, N, p, nx, nk, seed)
    (2, 1.0, 5, 30, 25, 1),
    (2, 2.0, 3, 40, 30, 2),
    (2, 16.0, 5, 200, 150, 3),
    (2, 64.0, 7, 500, 400, 4),
    (2, 32.0, 9, 300, 300, 5),
    (3, 4.0, 3, 200, 150, 6),
    (3, 8.0, 5, 400, 300, 7),
    (3, 4.0, 7, 150, 120, 8),
    # N not a power of two: leaves N / 2^L wide, a unit-modulus factor per output tile
    (2, 24.0, 5, 300, 250, 9),
    (2, 0.75, 5, 30, 25, 10),
    (2, 100.5, 7, 600, 500, 11),
    (3, 12.0, 5, 400, 300, 12),
    (3, 6.0, 3, 200, 200, 13),
]


@pytest.mark.parametrize("dim,N,p,nx,nk,seed", SMALL)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_random_points_match_oracle(dim, N, p, nx, nk, seed, prec):
    inst = w.small_random(dim, N, p, nx, nk, seed, edge_fraction=0.2)
    f = inst.sources()[0]
    ref = ob.butterfly(inst.x, inst.k, f, N, p)
    got = _fwd(inst, f, prec)
    assert rel_l2(got, ref) < (TOL64 if prec == "fp64" else tol32(p))


@pytest.mark.parametrize("N,p", [(256.0, 5), (256.0, 7), (1024.0, 7), (512.0, 9), (700.0, 7), (1500.3, 5)])
def test_curves_match_oracle_and_band(N, p):
    x = w.sample_curve(w.circle_curve(), N)
    k = w.sample_curve(w.perturbed_ellipse_curve(), N)
    inst = w.Instance("c", 2, N, p, x, k)
    f = inst.sources()[0]
    ref = ob.butterfly(x, k, f, N, p)
    u64 = _fwd(inst, f, "fp64")
    u32 = _fwd(inst, f, "fp32", torch.complex64)
    assert rel_l2(u64, ref) < TOL64
    assert rel_l2(u32, ref) < tol32(p)
    assert rel_l2(u32, u64) < tol32(p)
    eps = rel_l2(u64, direct(x, k, f, N))
    assert eps < 2 * BANDS[(2, p)][1]


def test_circle256_fp64_configuration():
    inst = w.circle256()
    f = inst.sources(dtype=np.complex128)[0]
    ref = ob.butterfly(inst.x, inst.k, f, inst.N, inst.p)
    u = _fwd(inst, f, "fp64")
    assert rel_l2(u, ref) < TOL64
    assert rel_l2(u, direct(inst.x, inst.k, f, inst.N)) < 2 * BANDS[(2, 5)][1]


@pytest.mark.parametrize("p", [5, 7])
def test_sphere_3d(p):
    N = 16.0
    x = w.fibonacci_sphere(N)
    inst = w.Instance("s", 3, N, p, x, x.copy())
    f = inst.sources()[0]
    ref = ob.butterfly(x, x, f, N, p)
    assert rel_l2(_fwd(inst, f, "fp64"), ref) < TOL64
    assert rel_l2(_fwd(inst, f, "fp32", torch.complex64), ref) < tol32(p)


def test_many_points_in_one_leaf_and_ragged():
    # 700 sources in one unit leaf, 3 elsewhere; targets everywhere, some at N.
    rng = np.random.default_rng(3)
    N = 64.0
    k = np.concatenate([rng.uniform(10.0, 11.0, (700, 2)), rng.uniform(0, N, (3, 2))])
    x = w.random_points(257, N, 2, 4, edge_fraction=0.3)
    inst = w.Instance("r", 2, N, 5, x, k)
    f = inst.sources()[0]
    ref = ob.butterfly(x, k, f, N, 5)
    assert rel_l2(_fwd(inst, f, "fp64"), ref) < TOL64
    assert rel_l2(_fwd(inst, f, "fp32"), ref) < tol32(5)


def test_single_point_each_side():
    inst = w.Instance("one", 2, 128.0, 7, np.array([[3.25, 100.5]]), np.array([[128.0, 0.0]]))
    f = np.array([1.0 - 2.0j])
    ref = ob.butterfly(inst.x, inst.k, f, inst.N, 7)
    assert rel_l2(_fwd(inst, f, "fp64"), ref) < TOL64


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_multiple_rhs_and_io_dtypes(prec):
    inst = w.small_random(2, 128.0, 5, 600, 500, 11)
    f = inst.sources(nrhs=3)
    ref = ob.butterfly(inst.x, inst.k, f, inst.N, 5)
    tol = TOL64 if prec == "fp64" else tol32(5)
    u128 = _fwd(inst, f, prec, torch.complex128)
    u64 = _fwd(inst, f, prec, torch.complex64)
    for r in range(3):
        assert rel_l2(u128[r], ref[r]) < tol
        assert rel_l2(u64[r], ref[r]) < (1e-6 if prec == "fp32" else 1e-6)
    single = _fwd(inst, f[1], prec)
    assert rel_l2(single, u128[1]) < 1e-14          # RHS are independent


def test_deterministic():
    inst = w.small_random(2, 256.0, 7, 2000, 2000, 12)
    f = inst.sources()[0]
    P = _plan(inst, "fp32")
    a = P.forward(_gpu(f, torch.complex64))
    b = P.forward(_gpu(f, torch.complex64))
    assert torch.equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_direct_sum_on_gpu(prec):
    inst = w.small_random(3, 32.0, 5, 700, 900, 13)
    f = inst.sources(nrhs=2)
    P = _plan(inst, prec, nrhs=2)
    u = P.direct(_gpu(f)).cpu().numpy()
    ref = direct(inst.x, inst.k, f, inst.N)
    assert rel_l2(u, ref) < (1e-12 if prec == "fp64" else 2e-6)
    uu = w.gaussian_sources(inst.x.shape[0], nrhs=2, seed=5)
    fa = P.direct(_gpu(uu), adjoint=True).cpu().numpy()
    assert rel_l2(fa, direct_adjoint(inst.x, inst.k, uu, inst.N)) < (1e-12 if prec == "fp64" else 2e-6)


def test_execute_host_matches_device():
    inst = w.small_random(2, 64.0, 7, 300, 250, 14)
    f = inst.sources()[0].astype(np.complex64)
    P = _plan(inst, "fp32")
    dev = P.forward(_gpu(f, torch.complex64)).cpu().numpy()
    host = P.execute_host(f)
    assert np.array_equal(dev, host)
    ua = P.execute_host(host, adjoint=True)
    assert np.array_equal(ua, P.adjoint(_gpu(host, torch.complex64)).cpu().numpy())


@pytest.mark.parametrize("dim,N,p", [(2, 4096.0, 7), (2, 2048.0, 5), (3, 64.0, 5)])
def test_events_path_matches_and_counts_launches(dim, N, p):
    # bfly_execute_events: one event before every launch (leaf, the recursive-step launches
    # of one or two stages each, final) and one after; same results as bfly_execute
    inst = w.small_random(dim, N, p, 600, 500, 21)
    f = _gpu(inst.sources()[0], torch.complex64)
    P = _plan(inst, "fp32")
    info = P.info()
    L, S = info["L"], info["steps"]
    assert S == len(P.steps()) and (-(-L // 3) if dim == 2 else L) <= S <= L
    for adjoint in (False, True):
        v = f if not adjoint else P.forward(f)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(S + 3)]
        for e in ev:
            e.record()
        got = P.with_events(v, ev, adjoint=adjoint)
        torch.cuda.synchronize()
        ref = P.adjoint(v) if adjoint else P.forward(v)
        assert torch.equal(got, ref)
        assert all(ev[i].elapsed_time(ev[i + 1]) >= 0.0 for i in range(S + 2))
    with pytest.raises(RuntimeError):
        P.with_events(f, [torch.cuda.Event(enable_timing=True) for _ in range(L + 3 + (S == L))])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_empty_sides(prec):
    # no sources: every potential is zero; no targets: an empty result; the adjoint mirrors
    from paper_0801_1524_gb300.plan import Batch, Plan
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    x = w.random_points(50, 64.0, 2, 1)
    none = np.zeros((0, 2))
    P = Plan(x, none, 64.0, 5, precision=prec, max_nrhs=2)
    u = P.forward(torch.zeros((2, 0), dtype=dt, device="cuda"), out=torch.full((2, 50), 7.0, dtype=dt, device="cuda"))
    assert u.shape == (2, 50) and torch.count_nonzero(u).item() == 0
    assert P.adjoint(torch.ones((2, 50), dtype=dt, device="cuda")).shape == (2, 0)
    uh = P.execute_host(np.zeros((1, 0), dtype=np.complex128))
    assert uh.shape == (1, 50) and not np.any(uh)
    Q = Plan(none, x, 64.0, 5, precision=prec)
    assert Q.forward(torch.ones(50, dtype=dt, device="cuda")).shape == (0,)
    g = Q.adjoint(torch.zeros(0, dtype=dt, device="cuda"))
    assert g.shape == (50,) and torch.count_nonzero(g).item() == 0
    torch.cuda.synchronize()
    # a batch with an empty member next to a regular one
    inst = w.small_random(2, 64.0, 5, 300, 200, 3)
    R = Plan(inst.x, inst.k, 64.0, 5, precision=prec)
    f = torch.as_tensor(inst.sources()[0], device="cuda").to(dt)
    B = Batch([P, R])
    us = B.forward([torch.zeros((1, 0), dtype=dt, device="cuda"), f.reshape(1, -1)])
    torch.cuda.synchronize()
    assert torch.count_nonzero(us[0]).item() == 0
    assert torch.equal(us[1].reshape(-1), R.forward(f))


@pytest.mark.parametrize("prec,dt", [("fp32", np.complex64), ("fp64", np.complex128)])
def test_execute_host_on_pinned_buffers(prec, dt):
    # pinned host buffers are read and written in place by the leaf and final steps; the
    # arithmetic is the same as on device buffers, so the results are identical
    inst = w.small_random(2, 128.0, 7, 700, 600, 15)
    P = _plan(inst, prec, nrhs=2)
    tdt = torch.complex64 if dt == np.complex64 else torch.complex128
    f_pin = torch.empty((2, inst.k.shape[0]), dtype=tdt).pin_memory()
    f_pin.copy_(torch.as_tensor(inst.sources(nrhs=2)))
    u_pin = torch.full((2, inst.x.shape[0]), 3.0, dtype=tdt).pin_memory()
    P.execute_host(f_pin.numpy(), out=u_pin.numpy())
    dev = P.forward(f_pin.to("cuda")).cpu()
    assert torch.equal(u_pin, dev)
    g_pin = torch.zeros((2, inst.k.shape[0]), dtype=tdt).pin_memory()
    P.execute_host(u_pin.numpy(), adjoint=True, out=g_pin.numpy())
    assert torch.equal(g_pin, P.adjoint(u_pin.to("cuda")).cpu())
    # pageable buffers take the staging copies: the same results
    assert np.array_equal(P.execute_host(f_pin.numpy().copy()), u_pin.numpy())


@pytest.mark.parametrize("dim,N,n,p", [(2, 2.0 ** 20, 120, 5), (2, 2.0 ** 16 + 0.5, 100, 7), (3, 2.0 ** 10, 60, 3),
                                       (2, 2.0 ** 30, 40, 3)])
def test_deep_trees(dim, N, n, p):
    # few points in a large domain: up to 30 levels, mostly single-box stages, every
    # launch of the recursive step with a handful of chunks
    # The oracle forms its phases 2 pi x.k/N from absolute coordinates (|x|, |k| <= N), so
    # its own FP64 rounding is about N eps relative (2.4e-7 at N = 2^30); the CUDA path
    # forms no phase beyond a unit leaf (exact offsets, operators independent of N).  The
    # FP64 comparison allows that rounding on top of the 1e-9 gate.
    inst = w.small_random(dim, N, p, n, n, 17, edge_fraction=0.2)
    f = inst.sources()[0]
    ref = ob.butterfly(inst.x, inst.k, f, N, p)
    u64 = _fwd(inst, f, "fp64")
    assert rel_l2(u64, ref) < TOL64 + 4 * N * np.finfo(float).eps
    assert rel_l2(_fwd(inst, f, "fp32", torch.complex64), ref) < tol32(p)
    assert rel_l2(_fwd(inst, f, "fp32", torch.complex64), u64) < tol32(p)


def test_coincident_points():
    # repeated targets and sources (the same coordinates several times, some on box edges)
    rng = np.random.default_rng(21)
    N = 256.0
    base_x = w.random_points(60, N, 2, 22, edge_fraction=0.3)
    base_k = w.random_points(50, N, 2, 23, edge_fraction=0.3)
    x = base_x[rng.integers(0, 60, 400)]
    k = base_k[rng.integers(0, 50, 300)]
    inst = w.Instance("dup", 2, N, 7, x, k)
    f = inst.sources()[0]
    ref = ob.butterfly(x, k, f, N, 7)
    u64 = _fwd(inst, f, "fp64")
    assert rel_l2(u64, ref) < TOL64
    assert rel_l2(_fwd(inst, f, "fp32", torch.complex64), ref) < tol32(7)
    # equal targets get equal potentials
    first = {}
    for i, row in enumerate(map(tuple, x)):
        if row in first:
            assert u64[i] == u64[first[row]]
        else:
            first[row] = i
