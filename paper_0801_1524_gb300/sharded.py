"""One transform sharded over ranks (one GPU each): the butterfly sweep of Sec. 2.2 cut at a
middle stage t_mid.

Stage t pairs the T_X boxes A of level L - t with the T_K boxes B of level t, and the
recursive step builds stage t from stage t + 1 through the children of B and the parent
of A.  So

* stages L .. t_mid need, for a box B of level >= t_mid, only the sources under B: the
  ranks split the T_K boxes of level t_mid (contiguous runs of the Morton order, balanced
  by source count); rank r runs the leaf step and the recursive step down to stage t_mid
  on its sources, for every A;
* stages t_mid - 1 .. 0 need, for a box A of level > L - t_mid, only the charges of its
  ancestor of level a0 = L - t_mid: the ranks split the T_X boxes of level a0 the same
  way (balanced by target count); rank r runs the rest of the sweep and the final step for
  its targets, for every B;
* in between, one exchange: rank q sends to rank r the stage-t_mid tiles (A in r's T_X
  boxes) x (B in q's T_K boxes); rank r puts them side by side in B.  That is one level's
  charges in all, sent once (an all-to-all of point-to-point messages, no collective on
  the compute path).

ShardLayout is the host-side partition (from a host-only plan of all points);
pack/assemble/exchange_p2p are the exchange; ShardedTransform runs one rank on its GPU
(bfly_execute_to_stage, the exchange, bfly_execute_from_stage).  The adjoint runs the same
way backwards: the ranks of T_X boxes take their targets up to stage t_mid, the exchange
is transposed (pack_adjoint/assemble_adjoint: blocks split in B, joined in A), and the
ranks of T_K boxes finish with the leaf step's transpose for their sources.
"""
from __future__ import annotations

import math

import numpy as np

from .plan import Plan


def _scale_and_levels(N: float):
    """L = ceil(log2 N) (0 for N <= 1) and the point scale sqrt(2^L / N) of the plan."""
    L = 0 if not N > 1.0 else int(math.ceil(math.log2(N) - 1e-12))
    rho = math.ldexp(N, -L)
    return L, (1.0 if rho == 1.0 else math.sqrt(math.ldexp(1.0, L) / N))


def box_of(pts, N: float, level: int) -> np.ndarray:
    """Box index per axis of every point at tree level `level`, by the plan's rule: leaf
    min(floor(s v), 2^L - 1) per coordinate (s the point scale), then the ancestor."""
    L, s = _scale_and_levels(float(N))
    u = np.asarray(pts, dtype=np.float64) * s if s != 1.0 else np.asarray(pts, dtype=np.float64)
    leaf = np.minimum(np.floor(u).astype(np.int64), (1 << L) - 1)
    return leaf >> (L - level)


def _split_runs(boxes, point_boxes, world):
    """Contiguous runs of `boxes` (Morton order) for `world` ranks, balanced by the number of
    points in each box: returns the run bounds [world + 1] and each point's rank."""
    pos = {tuple(b): i for i, b in enumerate(boxes)}
    which = np.array([pos[tuple(b)] for b in point_boxes], dtype=np.int64) if len(point_boxes) else \
        np.zeros(0, dtype=np.int64)
    count = np.bincount(which, minlength=len(boxes))
    cum = np.concatenate([[0], np.cumsum(count)])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world):
        # the first box whose points start at or after r/world of all points
        bounds.append(max(bounds[-1], int(np.searchsorted(cum[:-1], r * total / world, side="left"))))
    bounds.append(len(boxes))
    owner_of_box = np.zeros(len(boxes), dtype=np.int64)
    for r in range(world):
        owner_of_box[bounds[r]:bounds[r + 1]] = r
    return np.array(bounds), owner_of_box[which] if len(which) else which


class ShardLayout:
    """The partition of one transform (targets x, sources k, domain N, p) over `world` ranks."""

    def __init__(self, x, k, N: float, p: int, world: int, stages: int = 0, t_mid: int | None = None):
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.k = np.ascontiguousarray(k, dtype=np.float64)
        self.N, self.p, self.world, self.stages = float(N), int(p), int(world), int(stages)
        H = Plan(self.x, self.k, self.N, self.p, host_only=True, stages=stages)
        self.L = H.info()["L"]
        self.dim = self.x.shape[1]
        if t_mid is None:
            bounds = [self.L] + [t - lev + 1 for t, lev in H.steps()]
            t_mid = min(bounds, key=lambda t: (abs(t - self.L / 2.0), -t))
        self.t_mid = int(t_mid)
        self.a0 = self.L - self.t_mid
        # T_K boxes of level t_mid and T_X boxes of level a0, in the plan's (Morton) order
        self.kboxes = H.boxes("k", self.t_mid)
        self.xboxes = H.boxes("x", self.a0)
        self.kb, src_rank = _split_runs(self.kboxes, box_of(self.k, self.N, self.t_mid), world)
        self.xb, tgt_rank = _split_runs(self.xboxes, box_of(self.x, self.N, self.a0), world)
        # caller indices of every rank's sources and targets (increasing)
        self.sources = [np.nonzero(src_rank == r)[0] for r in range(world)]
        self.targets = [np.nonzero(tgt_rank == r)[0] for r in range(world)]

    def n_kboxes(self, r):
        return int(self.kb[r + 1] - self.kb[r])

    def n_xboxes(self, r):
        return int(self.xb[r + 1] - self.xb[r])

    def tile_stride(self, precision: str) -> int:
        pd = self.p ** self.dim
        return pd if precision == "fp64" else pd + (pd & 1)


def pack(layout: ShardLayout, rank: int, charges):
    """The blocks rank `rank` sends: charges [nrhs, nA (all of level a0), nB (its boxes of
    level t_mid), TS] -> for every rank q the rows A of q's boxes, [nrhs, nA_q, nB, TS]."""
    return [charges[:, layout.xb[q]:layout.xb[q + 1]].contiguous() for q in range(layout.world)]


def assemble(layout: ShardLayout, rank: int, received):
    """Rank `rank`'s stage-t_mid input from the blocks of every rank q, [nrhs, nA_r, nB_q,
    TS] -> [nrhs, nA_r, nB (all of level t_mid), TS] (q's boxes are the run kb[q]:kb[q+1])."""
    import torch
    return torch.cat(list(received), dim=2).contiguous()


def pack_adjoint(layout: ShardLayout, rank: int, charges):
    """The adjoint sweep's blocks of rank `rank`: charges [nrhs, nA_r, nB (all of level
    t_mid), TS] -> for every rank q the columns B of q's boxes, [nrhs, nA_r, nB_q, TS]."""
    return [charges[:, :, layout.kb[q]:layout.kb[q + 1]].contiguous() for q in range(layout.world)]


def assemble_adjoint(layout: ShardLayout, rank: int, received):
    """Rank `rank`'s stage-t_mid input of the adjoint sweep: the blocks [nrhs, nA_q, nB_r,
    TS] of every rank q side by side in A -> [nrhs, nA (all of level a0), nB_r, TS]."""
    import torch
    return torch.cat(list(received), dim=1).contiguous()


def exchange_p2p(sends, recv_shapes, rank: int, world: int, dist, group=None):
    """Point-to-point exchange: sends[q] goes to rank q, the block from rank q (shape
    recv_shapes[q]) is returned at position q; the own block is kept in place."""
    import torch
    recvs = [None] * world
    ops = []
    for q in range(world):
        if q == rank:
            recvs[q] = sends[q]
            continue
        recvs[q] = torch.empty(recv_shapes[q], dtype=sends[q].dtype, device=sends[q].device)
        if sends[q].numel():
            ops.append(dist.P2POp(dist.isend, sends[q], q, group))
        if recvs[q].numel():
            ops.append(dist.P2POp(dist.irecv, recvs[q], q, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return recvs


class ShardedTransform:
    """Rank `rank` of the sharded forward transform on its GPU: the first part of the sweep
    for its sources, the exchange, the second part for its targets.  Input: the sources
    layout.sources[rank] ([nrhs, n] in that order); output: the targets
    layout.targets[rank]."""

    def __init__(self, layout: ShardLayout, rank: int, precision: str = "fp32", max_nrhs: int = 1):
        self.layout, self.rank, self.precision = layout, int(rank), precision
        L = layout
        self.up = Plan(L.x, L.k[L.sources[rank]], L.N, L.p, precision=precision, max_nrhs=max_nrhs,
                       stages=L.stages)
        self.lo = Plan(L.x[L.targets[rank]], L.k, L.N, L.p, precision=precision, max_nrhs=max_nrhs,
                       stages=L.stages)
        self.ts = L.tile_stride(precision)
        for pl in (self.up, self.lo):
            if L.t_mid not in pl.boundaries():
                raise ValueError(f"stage {L.t_mid} is not a launch boundary of a rank's plan; build the "
                                 "layout with stages=1")

    def upper(self, f_local):
        """Stage-t_mid charges of this rank's sources, [nrhs, nA, nB_r, TS]."""
        L = self.layout
        c = self.up.to_stage(f_local, L.t_mid)
        return c.reshape(c.shape[0], len(L.xboxes), L.n_kboxes(self.rank), self.ts)

    def lower(self, charges, out=None):
        """Potentials of this rank's targets from its stage-t_mid input [nrhs, nA_r, nB, TS]."""
        return self.lo.from_stage(charges.reshape(charges.shape[0], -1), self.layout.t_mid, out=out)

    def recv_shapes(self, nrhs):
        L = self.layout
        return [(nrhs, L.n_xboxes(self.rank), L.n_kboxes(q), self.ts) for q in range(L.world)]

    def forward(self, f_local, dist, group=None):
        c = self.upper(f_local)
        got = exchange_p2p(pack(self.layout, self.rank, c), self.recv_shapes(c.shape[0]), self.rank,
                           self.layout.world, dist, group)
        return self.lower(assemble(self.layout, self.rank, got))

    # ---- the adjoint (the exact conjugate transpose: the sweep run backwards, T_X to T_K)
    def upper_adjoint(self, u_local):
        """Stage-t_mid charges of the adjoint sweep from this rank's targets (the final
        step's transpose and the adjoint sweep up to t_mid), [nrhs, nA_r, nB, TS]."""
        L = self.layout
        c = self.lo.to_stage(u_local, L.t_mid, adjoint=True)
        return c.reshape(c.shape[0], L.n_xboxes(self.rank), len(L.kboxes), self.ts)

    def lower_adjoint(self, charges, out=None):
        """This rank's sources from its stage-t_mid input of the adjoint [nrhs, nA, nB_r, TS]."""
        return self.up.from_stage(charges.reshape(charges.shape[0], -1), self.layout.t_mid, out=out, adjoint=True)

    def recv_shapes_adjoint(self, nrhs):
        L = self.layout
        return [(nrhs, L.n_xboxes(q), L.n_kboxes(self.rank), self.ts) for q in range(L.world)]

    def adjoint(self, u_local, dist, group=None):
        c = self.upper_adjoint(u_local)
        got = exchange_p2p(pack_adjoint(self.layout, self.rank, c), self.recv_shapes_adjoint(c.shape[0]),
                           self.rank, self.layout.world, dist, group)
        return self.lower_adjoint(assemble_adjoint(self.layout, self.rank, got))
