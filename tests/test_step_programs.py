"""Host compiler of the recursive step (Sec. 2.2 step 3) checked on the CPU.

The chunk programs the library compiles (bfly_plan_program) are executed here by a plain
numpy interpreter that follows their documented format: per pass, every item applies its
operator along the pass's axis to one or two source tiles of the previous pass and sums
them.  The operators are random matrices, so the checks hold for any operator values:

* fusing stages into one launch changes nothing: the programs of the default plan (up to
  three stages per launch in 2D, the middle stages never leaving shared memory) give the
  same stage-0 charges as the one-stage programs (BFLY_FLAG_ONE_STAGE) of the same points;
* the adjoint programs are the adjoint: <F x, y> = <x, F^H y> with the conjugate-
  transposed operators, F the whole forward sweep of the recursive step.
"""
import numpy as np
import pytest

from paper_0801_1524_gb300 import native
from paper_0801_1524_gb300 import workloads as w
from paper_0801_1524_gb300.plan import Plan

ORUN = np.dtype([("start", "<i4"), ("slot", "<u2"), ("count", "<u2")])


def _apply(M, x, axis):
    """y[.., m, ..] = sum_l M[m, l] x[.., l, ..] along `axis` of the tile."""
    return np.moveaxis(np.tensordot(M, x, axes=([1], [axis])), 0, axis)


def run_program(prog, dim, p, tiles_in, n_out, ops):
    """Executes one launch's chunk program on tiles_in [n_in][p]*dim; returns [n_out][p]*dim."""
    out = np.full((n_out,) + (p,) * dim, np.nan + 0j)
    written = np.zeros(n_out, dtype=bool)
    blob = prog["blob"]
    runs = prog["runs"].view(ORUN)
    for c in prog["chunks"]:
        blob_off, blob_bytes, run_off, n_runs, n_in, n_pass = (int(v) for v in c[:6])
        hdr = blob[blob_off:blob_off + 64].view(np.int32)
        NP, n_oruns = int(hdr[0]), int(hdr[2])
        assert NP == n_pass and NP % dim == 0 and int(hdr[1]) == n_in
        n_item = [int(v) for v in hdr[4:4 + NP]]
        n_two = [int(v) for v in hdr[10:10 + NP]]
        items = blob[blob_off + 64:blob_off + 64 + 8 * sum(n_item)].view(np.uint16).reshape(-1, 4)
        obeg = blob_off + 64 + 8 * sum(n_item)
        oruns = blob[obeg:obeg + 8 * n_oruns].view(ORUN)
        # inputs: slot <- global tile, run by run
        src = {}
        for rn in runs[run_off:run_off + n_runs]:
            for q in range(int(rn["count"])):
                src[int(rn["slot"]) + q] = tiles_in[int(rn["start"]) + q]
        assert sorted(src) == list(range(n_in))
        off = 0
        for j in range(NP):
            dst = {}  # a pass reads only what the previous pass wrote
            for i, (s0, s1, d, op) in enumerate(items[off:off + n_item[j]]):
                y = _apply(ops[int(op) & 3], src[int(s0)], j % dim)
                assert (s1 != 0xFFFF) == (i < n_two[j])
                if s1 != 0xFFFF:
                    y = y + _apply(ops[(int(op) >> 2) & 3], src[int(s1)], j % dim)
                assert int(d) not in dst
                dst[int(d)] = y
            off += n_item[j]
            src = dst
        for rn in oruns:
            for q in range(int(rn["count"])):
                g = int(rn["start"]) + q
                assert not written[g]
                out[g] = src[int(rn["slot"]) + q]
                written[g] = True
    assert written.all()
    return out


def sweep(P, x, ops, adjoint=False):
    """The recursive step of every launch, forward (stage L -> 0) or adjoint (0 -> L)."""
    dim, p = P.dim, P.p
    pairs = {t: a * b for t, a, b in P.stages()}
    steps = P.steps()
    order = range(len(steps)) if not adjoint else range(len(steps) - 1, -1, -1)
    for s in order:
        t, lev = steps[s]
        n_out = pairs[t - lev + 1] if not adjoint else pairs[t + 1]
        x = run_program(P.program(s, adjoint), dim, p, x, n_out, ops)
    return x


def _random_ops(rng, p):
    return rng.standard_normal((4, p, p)) + 1j * rng.standard_normal((4, p, p))


CASES = [(2, 64.0, 5, 150, 120, 1), (2, 256.0, 7, 300, 260, 2), (2, 128.0, 3, 200, 200, 3),
         (2, 96.0, 5, 180, 150, 4), (3, 16.0, 3, 150, 120, 5)]


@pytest.mark.parametrize("dim,N,p,nx,nk,seed", CASES)
def test_fused_steps_equal_one_stage_steps(dim, N, p, nx, nk, seed):
    inst = w.small_random(dim, N, p, nx, nk, seed, edge_fraction=0.3)
    fused = Plan(inst.x, inst.k, N, p, host_only=True)
    single = Plan(inst.x, inst.k, N, p, host_only=True, flags=native.BFLY_FLAG_ONE_STAGE)
    L = fused.info()["L"]
    assert single.steps() == [(t, 1) for t in range(L - 1, -1, -1)]
    if dim == 2:
        assert max(lev for _, lev in fused.steps()) > 1  # something is fused
    rng = np.random.default_rng(seed)
    ops = _random_ops(rng, p)
    n_in = fused.stages()[-1][1] * fused.stages()[-1][2]
    x = rng.standard_normal((n_in,) + (p,) * dim) + 1j * rng.standard_normal((n_in,) + (p,) * dim)
    a = sweep(fused, x, ops)
    b = sweep(single, x, ops)
    assert a.shape == b.shape
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-10 * np.abs(b).max())


@pytest.mark.parametrize("dim,N,p,nx,nk,seed", CASES[:3] + CASES[4:])
def test_adjoint_programs_are_the_adjoint(dim, N, p, nx, nk, seed):
    inst = w.small_random(dim, N, p, nx, nk, seed + 10, edge_fraction=0.3)
    P = Plan(inst.x, inst.k, N, p, host_only=True)
    rng = np.random.default_rng(seed + 10)
    ops = _random_ops(rng, p)
    opsH = np.conj(np.transpose(ops, (0, 2, 1)))
    st = P.stages()
    n_L, n_0 = st[-1][1] * st[-1][2], st[0][1] * st[0][2]
    shape = lambda n: (n,) + (p,) * dim
    x = rng.standard_normal(shape(n_L)) + 1j * rng.standard_normal(shape(n_L))
    y = rng.standard_normal(shape(n_0)) + 1j * rng.standard_normal(shape(n_0))
    Fx = sweep(P, x, ops)
    FHy = sweep(P, y, opsH, adjoint=True)
    lhs, rhs = np.vdot(y, Fx), np.vdot(FHy, x)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_planted_slot_error_is_caught():
    # the interpreter itself: a destination slot moved onto another one must fail
    inst = w.small_random(2, 64.0, 5, 120, 100, 7, edge_fraction=0.3)
    P = Plan(inst.x, inst.k, 64.0, 5, host_only=True)
    prog = P.program(0)
    c = prog["chunks"][0]
    items = prog["blob"][int(c[0]) + 64:].view(np.uint16)
    hdr = prog["blob"][int(c[0]):int(c[0]) + 64].view(np.int32)
    if hdr[4] < 2:
        pytest.skip("first pass has a single item")
    items[2] = items[6]  # item 0 now writes item 1's destination
    rng = np.random.default_rng(0)
    st = P.stages()
    n_in = st[-1][1] * st[-1][2]
    t, lev = P.steps()[0]
    x = rng.standard_normal((n_in, 5, 5)) + 0j
    with pytest.raises(AssertionError):
        run_program(prog, 2, 5, x, {t: a * b for t, a, b in st}[t - lev + 1], _random_ops(rng, 5))
