"""CPU-only checks of the C ABI: the library builds, loads and exports every function
include/bfly.h declares; argument validation; the host plan (trees and stage sizes)
against the oracle's independent tree construction.  No kernel is launched."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle.butterfly as ob
from paper_0801_1524_gb300 import native
from paper_0801_1524_gb300 import workloads as w
from paper_0801_1524_gb300.plan import Plan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "bfly.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bfly_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    lib = native.load()
    names = header_functions()
    assert "bfly_execute" in names and len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(native.SIGNATURES)
    assert lib.bfly_version().decode().startswith("bfly")


def _create(dim=2, N=16.0, x=None, k=None, p=5, flags=native.BFLY_FLAG_HOST_ONLY, prec=1):
    lib = native.load()
    if x is None:
        x = w.random_points(10, 16.0, dim, 1)
    if k is None:
        k = w.random_points(10, 16.0, dim, 2)
    x = np.ascontiguousarray(x, float)
    k = np.ascontiguousarray(k, float)
    h = ctypes.c_void_p()
    o = native.Opts()
    o.prec, o.max_nrhs, o.flags = prec, 1, flags
    st = lib.bfly_plan_create(ctypes.byref(h), dim, float(N), x.shape[0], x.ctypes.data,
                              k.shape[0], k.ctypes.data, p, ctypes.byref(o))
    if st == 0:
        lib.bfly_plan_destroy(h)
    return st, lib.bfly_last_error().decode()


@pytest.mark.parametrize("kw,status", [
    (dict(dim=4), 1), (dict(dim=1), 1), (dict(p=2), 1), (dict(p=11), 1), (dict(p=4), 4),
    (dict(N=-3.0), 1), (dict(N=0.0), 1), (dict(N=float("nan")), 1), (dict(N=float("inf")), 1),
    (dict(x=np.array([[1.0, 17.0]])), 1), (dict(k=np.array([[-0.5, 1.0]])), 1),
    (dict(k=np.array([[np.nan, 1.0]])), 1), (dict(prec=7), 1),
])
def test_invalid_arguments_are_reported(kw, status):
    st, msg = _create(**kw)
    assert st == status and msg


def test_null_and_host_only_execution_rejected():
    lib = native.load()
    assert lib.bfly_plan_create(None, 2, 16.0, 1, None, 1, None, 5, None) == 1
    P = Plan(w.random_points(5, 16.0, 2, 1), w.random_points(5, 16.0, 2, 2), 16.0, 5, host_only=True)
    assert lib.bfly_execute(P._h, ctypes.c_void_p(8), ctypes.c_void_p(8), 1, 0, None) == 1
    assert "host-only" in lib.bfly_last_error().decode()
    assert lib.bfly_plan_stage(P._h, 99, ctypes.byref(ctypes.c_int64()), ctypes.byref(ctypes.c_int64())) == 1


@pytest.mark.parametrize("dim,N,p,nx,nk,seed", [
    (2, 1.0, 5, 7, 9, 1), (2, 64.0, 5, 300, 200, 2), (3, 16.0, 3, 400, 300, 3), (2, 2.0, 7, 20, 20, 4),
    # N not a power of two: leaves N / 2^L wide
    (2, 24.0, 5, 300, 200, 5), (3, 12.0, 3, 300, 300, 6), (2, 0.75, 5, 10, 10, 7), (2, 1000.5, 7, 400, 400, 8),
])
def test_stage_sizes_match_oracle_trees(dim, N, p, nx, nk, seed):
    inst = w.small_random(dim, N, p, nx, nk, seed, edge_fraction=0.3)
    P = Plan(inst.x, inst.k, N, p, host_only=True)
    ref = ob.pair_counts(inst.x, inst.k, N)
    got = {t: (a, b) for t, a, b in P.stages()}
    assert got == ref
    info = P.info()
    assert info["total_pairs"] == sum(a * b for a, b in ref.values())
    assert info["L"] == ob.levels_for(N)
    assert info["rho"] == N / 2.0 ** info["L"]
    assert 0.5 < info["rho"] <= 1.0 or N <= 1.0


def test_curve_workload_plan_counts():
    inst = w.curve8192()
    P = Plan(inst.x, inst.k, inst.N, inst.p, host_only=True)
    info = P.info()
    st = P.stages()
    # Sec. 2.2: stage t pairs nA(L-t) x nK(t), O(N) per stage, L = log2 N stages.
    assert info["L"] == 13 and len(st) == 14
    assert st[0][2] == 1 and st[-1][1] == 1
    assert all(a * b <= 12 * inst.N for _, a, b in st)
    assert info["tiles_written_fwd"] == sum(a * b for t, a, b in st if t < 13)
    assert info["plan_seconds"] < 5.0
    # stage 12 alone, then (11, 10, 9), (8, 7, 6), (5, 4, 3), (2, 1, 0): 5 launches
    assert P.steps() == [(12, 1), (11, 3), (8, 3), (5, 3), (2, 3)]


@pytest.mark.parametrize("dim,N,p", [(2, 1.0, 5), (2, 2.0, 5), (2, 4.0, 7), (2, 8.0, 7), (2, 16.0, 7),
                                     (2, 1000.5, 7), (3, 16.0, 5), (3, 12.0, 3)])
def test_recursive_step_launches(dim, N, p):
    # 2D: up to three stages per launch ((2, 1, 0), (5, 4, 3), .., the L mod 3 top stages
    # together; a group whose units exceed the shared-memory capacities is split);
    # 3D: one stage per launch.  Every program passed validation at plan creation.
    inst = w.small_random(dim, N, p, 200, 150, 9, edge_fraction=0.3)
    P = Plan(inst.x, inst.k, N, p, host_only=True)
    info = P.info()
    st = P.steps()
    L = info["L"]
    assert len(st) == info["steps"]
    assert (-(-L // 3) if dim == 2 else L) <= len(st) <= L
    t = info["L"] - 1
    for t0, lev in st:  # consecutive stages from L-1 down to 0
        assert t0 == t and 1 <= lev <= (3 if dim == 2 else 1)
        t -= lev
    assert t == -1
    bad = P._lib.bfly_plan_step(P._h, info["steps"], ctypes.byref(ctypes.c_int()), ctypes.byref(ctypes.c_int()))
    assert bad == 1  # BFLY_ERR_INVALID_ARG: step out of range


@pytest.mark.parametrize("nx,nk", [(0, 40), (40, 0), (0, 0)])
def test_empty_sides_are_accepted(nx, nk):
    x = w.random_points(nx, 64.0, 2, 1)
    k = w.random_points(nk, 64.0, 2, 2)
    P = Plan(x, k, 64.0, 5, host_only=True)
    info = P.info()
    assert (info["nx"], info["nk"]) == (nx, nk)
    # no non-empty box on an empty side: every stage pairs zero boxes with the other tree
    assert info["total_pairs"] == 0 and info["chunks_fwd"] == 0
    lib = native.load()
    h = ctypes.c_void_p()
    o = native.Opts()
    o.prec, o.max_nrhs, o.flags = 1, 1, native.BFLY_FLAG_HOST_ONLY
    assert lib.bfly_plan_create(ctypes.byref(h), 2, 64.0, nx, None, nk, None if nk == 0 else
                                np.ascontiguousarray(k).ctypes.data, 5, ctypes.byref(o)) == (1 if nx > 0 else 0)
    if h.value:
        lib.bfly_plan_destroy(h)


def test_program_export_sizes_and_errors():
    inst = w.small_random(2, 256.0, 7, 300, 260, 11, edge_fraction=0.3)
    P = Plan(inst.x, inst.k, 256.0, 7, host_only=True)
    lib, n = P._lib, ctypes.c_int64()
    for s in range(P.info()["steps"]):
        for adj in (0, 1):
            prog = P.program(s, bool(adj))
            nch = prog["chunks"].shape[0]
            assert nch >= 1 and prog["runs"].size % 8 == 0 and prog["blob"].size % 16 == 0
            # a partial copy fills only cap bytes and still reports the whole size
            buf = np.full(40, 0xAB, dtype=np.uint8)
            assert lib.bfly_plan_program(P._h, s, adj, 0, buf.ctypes.data, 32, ctypes.byref(n)) == 0
            assert n.value == nch * 32 and (buf[32:] == 0xAB).all()
            assert (buf[:32].view(np.int32) == prog["chunks"][0]).all()
    assert lib.bfly_plan_program(P._h, P.info()["steps"], 0, 0, None, 0, ctypes.byref(n)) == native.BFLY_ERR_INVALID_ARG
    assert lib.bfly_plan_program(P._h, 0, 0, 3, None, 0, ctypes.byref(n)) == native.BFLY_ERR_INVALID_ARG
    assert lib.bfly_plan_program(None, 0, 0, 0, None, 0, ctypes.byref(n)) == native.BFLY_ERR_INVALID_ARG


@pytest.mark.parametrize("dim,N,p", [(2, 1.0, 5), (2, 2.0, 5), (2, 16.0, 7), (2, 1000.5, 7), (3, 16.0, 5),
                                     (3, 12.0, 3)])
def test_dataflow_plans_build(dim, N, p):
    # BFLY_FLAG_DATAFLOW: the launch entries and the source lists of every chunk (and their
    # checks: every input tile written by a chunk of the step before, every chunk after its
    # sources) are built at plan creation, also for a host-only plan
    inst = w.small_random(dim, N, p, 200, 150, 9, edge_fraction=0.3)
    P = Plan(inst.x, inst.k, N, p, host_only=True, dataflow=True)
    info = P.info()
    assert info["dataflow"] == (1 if info["steps"] > 0 else 0)
    if dim == 2 and info["L"] > 1:
        assert info["stages_per_launch"] == 2     # the default with the flag in 2D
        Q = Plan(inst.x, inst.k, N, p, host_only=True, dataflow=True, stages=3)
        assert Q.info()["stages_per_launch"] == 3 and Q.info()["dataflow"] == 1
    plain = Plan(inst.x, inst.k, N, p, host_only=True, stages=info["stages_per_launch"])
    assert plain.steps() == P.steps() and plain.info()["dataflow"] == 0


@pytest.mark.parametrize("nx,nk", [(0, 40), (40, 0)])
def test_dataflow_with_an_empty_side(nx, nk):
    P = Plan(w.random_points(nx, 64.0, 2, 1), w.random_points(nk, 64.0, 2, 2), 64.0, 5, host_only=True,
             dataflow=True)
    assert P.info()["chunks_fwd"] == 0


def test_dataflow_refused_with_tensor_cores_and_groups():
    inst = w.small_random(2, 64.0, 7, 300, 300, 41)
    for prec in ("tc", "fp32g"):
        with pytest.raises(native.BflyError):
            Plan(inst.x, inst.k, inst.N, inst.p, precision=prec, max_nrhs=8, host_only=True, dataflow=True)
