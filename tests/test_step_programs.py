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

With the operators of the method (C^{(gamma,delta)} = W(delta) diag(phi_gamma) for the
rescaled charges), the same programs carry the oracle's stage-L charges to its stage-0
charges: the tile order, the child bits and the operator indices of the compiled
programs agree with the oracle's Sec. 2.2 step 3.
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


# ---- the compiled programs with the operators of the method, against the oracle

def _lagrange_w(p, tau):
    """w(tau) = G^{-1} v(tau), G_{ll'} = e^{2 pi i l l'/q^2}, v(tau)_l = e^{2 pi i l tau/q}:
    the weights that carry charges on a child grid to the parent grid (eq. M1)."""
    q = p - 1
    l = np.arange(p)
    G = np.exp(2j * np.pi * np.outer(l, l) / q ** 2)
    return np.linalg.solve(G, np.exp(2j * np.pi * l * tau / q))


def _method_ops(p):
    """C^{(gamma, delta)}[m][l] = w_m(tau_l) e^{2 pi i gamma tau_l}, tau_l = (delta + l/q)/2,
    for the rescaled charges g_m = e^{2 pi i a m/q} f_m; op = gamma * 2 + delta."""
    q = p - 1
    ops = np.zeros((4, p, p), dtype=np.complex128)
    for gamma in (0, 1):
        for delta in (0, 1):
            for l in range(p):
                tau = (delta + l / q) / 2
                ops[gamma * 2 + delta][:, l] = _lagrange_w(p, tau) * np.exp(2j * np.pi * gamma * tau)
    return ops


def _rescale(F, boxes, p):
    """g^{AB}_m = prod_d e^{2 pi i a_d m_d / q} f^{AB}_m, a the index of A along each axis."""
    q, dim = p - 1, boxes.shape[1]
    G = F.astype(np.complex128).copy()
    m = np.arange(p)
    for d in range(dim):
        ph = np.exp(2j * np.pi * np.outer(boxes[:, d], m) / q)  # [nA, p]
        shape = [F.shape[0], 1] + [1] * dim
        shape[2 + d] = p
        G *= ph.reshape(shape)
    return G


def _to_plan_order(F, o_boxes_A, o_boxes_B, P, L, t):
    """Oracle tiles F[iA, iB] (lexicographic boxes) -> the plan's tile order iA * nB + iB."""
    pa, pb = P.boxes("x", L - t), P.boxes("k", t)
    ia = {tuple(b): i for i, b in enumerate(o_boxes_A)}
    ib = {tuple(b): i for i, b in enumerate(o_boxes_B)}
    ra = np.array([ia[tuple(b)] for b in pa])
    rb = np.array([ib[tuple(b)] for b in pb])
    return F[ra][:, rb].reshape((len(pa) * len(pb),) + F.shape[2:])


@pytest.mark.parametrize("dim,N,p,nx,nk,seed,flags", [
    (2, 64.0, 5, 150, 120, 31, 0), (2, 200.0, 7, 260, 240, 32, 0), (2, 64.0, 5, 150, 120, 31, 8),
    (3, 8.0, 3, 120, 100, 33, 0), (2, 0.75 * 128, 5, 160, 150, 34, 0)])
def test_programs_reproduce_the_oracle_stage_charges(dim, N, p, nx, nk, seed, flags):
    # stage L charges of the oracle (rescaled, in the plan's tile order) through every
    # compiled launch with the operators of the method give the oracle's stage-0 charges
    import oracle.butterfly as ob
    inst = w.small_random(dim, N, p, nx, nk, seed, edge_fraction=0.3)
    f = inst.sources()[0].astype(np.complex128)
    TX, TK, L, F = ob.stage_charges(inst.x, inst.k, f, N, p)
    P = Plan(inst.x, inst.k, N, p, host_only=True, flags=flags)
    assert P.info()["L"] == L
    gL = _to_plan_order(_rescale(F[L], TX.boxes[0], p), TX.boxes[0], TK.boxes[L], P, L, L)
    g0 = sweep(P, gL, _method_ops(p))
    ref = _to_plan_order(_rescale(F[0], TX.boxes[L], p), TX.boxes[L], TK.boxes[0], P, L, 0)
    # the oracle's charges come from FP64 LU solves of the matching systems, each
    # accurate to about cond(G)^dim * eps (G ill-conditioned: 4e2 at p = 5, 2e5 at
    # p = 7); a wiring mistake in the programs would be of the charges' own size
    q = p - 1
    l = np.arange(p)
    cond = np.linalg.cond(np.exp(2j * np.pi * np.outer(l, l) / q ** 2)) ** dim
    err = np.abs(g0 - ref).max() / np.abs(ref).max()
    assert err < 1e-9 + 20 * np.finfo(float).eps * cond, (err, cond)


@pytest.mark.parametrize("mistake", ["gamma_delta_swapped", "operators_transposed", "charges_not_rescaled"])
def test_planted_operator_mistakes_fail_the_oracle_check(mistake):
    import oracle.butterfly as ob
    inst = w.small_random(2, 64.0, 5, 150, 120, 31, edge_fraction=0.3)
    f = inst.sources()[0].astype(np.complex128)
    TX, TK, L, F = ob.stage_charges(inst.x, inst.k, f, 64.0, 5)
    P = Plan(inst.x, inst.k, 64.0, 5, host_only=True)
    ops = _method_ops(5)
    gL = _to_plan_order(_rescale(F[L], TX.boxes[0], 5), TX.boxes[0], TK.boxes[L], P, L, L)
    ref = _to_plan_order(_rescale(F[0], TX.boxes[L], 5), TX.boxes[L], TK.boxes[0], P, L, 0)
    if mistake == "gamma_delta_swapped":
        ops = ops[[0, 2, 1, 3]]
    elif mistake == "operators_transposed":
        ops = np.transpose(ops, (0, 2, 1))
    else:
        ref = _to_plan_order(F[0].astype(np.complex128), TX.boxes[L], TK.boxes[0], P, L, 0)
    g0 = sweep(P, gL, ops)
    assert np.abs(g0 - ref).max() / np.abs(ref).max() > 0.1


def _pairwise_sweep(TX, TK, L, gL, ops, dim):
    """The recursive step pair by pair on the oracle's trees (no programs, no fusion, no
    sum factorisation): g^{AB} = sum_c (x)_d C^{(gamma_d(A), delta_d(Bc))} g^{A'Bc} for
    every stage t = L-1 .. 0, tiles indexed [iA, iB] in the oracle's box order."""
    g = gL
    for t in range(L - 1, -1, -1):
        A, Ap, B, Bc = TX.boxes[L - t], TX.boxes[L - t - 1], TK.boxes[t], TK.boxes[t + 1]
        ia = {tuple(b): i for i, b in enumerate(Ap)}
        ib = {tuple(b): i for i, b in enumerate(B)}
        kids = {}
        for j, c in enumerate(Bc):
            kids.setdefault(ib[tuple(c // 2)], []).append(j)
        out = np.zeros((len(A), len(B)) + g.shape[2:], dtype=np.complex128)
        for i, a in enumerate(A):
            ip = ia[tuple(a // 2)]
            for jb, js in kids.items():
                for jc in js:
                    y = g[ip, jc]
                    for d in range(dim):
                        y = _apply(ops[(a[d] & 1) * 2 + (Bc[jc][d] & 1)], y, d)
                    out[i, jb] += y
        g = out
    return g


@pytest.mark.parametrize("dim,N,p,nx,nk,seed,flags", [
    (2, 200.0, 7, 260, 240, 32, 0), (2, 128.0, 9, 200, 180, 35, 0), (2, 200.0, 7, 260, 240, 32, 8),
    (3, 8.0, 5, 120, 100, 36, 0), (2, 0.75 * 128, 7, 160, 150, 34, 0)])
def test_programs_equal_the_pairwise_recursion(dim, N, p, nx, nk, seed, flags):
    # the same operators of the method on both sides, so that the conditioning of the
    # matching systems drops out: the compiled (fused, sum-factorised) programs must give
    # the pairwise recursion's stage-0 charges to rounding, and a 1e-6 change of one
    # operator must be seen
    import oracle.butterfly as ob
    inst = w.small_random(dim, N, p, nx, nk, seed, edge_fraction=0.3)
    f = inst.sources()[0].astype(np.complex128)
    TX, TK, L, F = ob.stage_charges(inst.x, inst.k, f, N, p)
    P = Plan(inst.x, inst.k, N, p, host_only=True, flags=flags)
    ops = _method_ops(p)
    gL_o = _rescale(F[L], TX.boxes[0], p)
    ref = _to_plan_order(_pairwise_sweep(TX, TK, L, gL_o, ops, dim), TX.boxes[L], TK.boxes[0], P, L, 0)
    gL = _to_plan_order(gL_o, TX.boxes[0], TK.boxes[L], P, L, L)
    scale = np.abs(ref).max()
    err = np.abs(sweep(P, gL, ops) - ref).max() / scale
    assert err < 1e-12, err
    planted = ops.copy()
    planted[3] *= 1.0 + 1e-6
    err_planted = np.abs(sweep(P, gL, planted) - ref).max() / scale
    assert err_planted > 1e-8, err_planted
