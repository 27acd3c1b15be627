"""Oracle — test infrastructure only (tests, the smoke check and the benchmark's CPU
baseline may use it; the product path never does).

The butterfly algorithm of Sec. 2.2 written out step by step in float64 numpy, in the
paper's notation, with nothing precomputed or fused:

  Step 1  build T_X and T_K: boxes of width w_s = N / 2^s at levels s = 0..L, leaves
          of unit width (N = 2^L), non-empty boxes only (Sec. 2.2 operation count).
  Step 2  for each leaf B of T_K, the check potentials u^{A0 B} at the grid x^{A0}_l of
          the root A0 of T_X by direct summation over the sources in B, then the
          equivalent charges f^{A0 B} on the grid k^B_l from M f = u (Sec. 2.1).
  Step 3  for t = L-1 .. 0, every B of T_K at level t and every A of T_X at level L-t:
          u^{AB}_l = sum_c sum_l' exp(2 pi i x^A_l . k^{Bc}_l' / N) f^{A'Bc}_l'
          (Sec. 2.1, Fig. 1: A' the parent of A, Bc the children of B), then M f = u.
  Step 4  for each leaf A of T_X and target x_i in A:
          u_i = sum_l exp(2 pi i x_i . k^{B0}_l / N) f^{A B0}_l, B0 the root of T_K.

Grids (Sec. 2.1): k^B_l = c^B + l w^B/(p-1) and x^A_l = c^A + l w^A/(p-1), l in
{0..p-1}^d, c the lower corner of the box.  The matrices M (matching) and E (evaluation)
are built entry by entry from these grid coordinates.  By default they are used in the
Kronecker form the paper states (M = M_1 (x) M_2, E = E_1 (x) E_2, inverses taken factor
by factor); `dense=True` builds the full p^d x p^d matrices instead, for small cases.
The paper's further factorisation of M_1 and E_1 into diagonal x G x diagonal and
diagonal x H x diagonal (eqs. M1 and E1) is deliberately not used here.

Readings where the paper is silent: a point on a box edge belongs to the box with the
larger index, except at the far edge N (index clamped to 2^s - 1); boxes of a level are
the non-empty ones; a missing child of B contributes nothing; the matching systems are
solved by LU with partial pivoting (numpy.linalg.solve).  N not a power of two (the
paper's setting has unit leaves, N = 2^L): with L = ceil(log2 N) and rho = N / 2^L,
x.k/N = x'.k'/2^L for x' = x s, k' = k s, s = sqrt(2^L / N), so the transform is the one
of N' = 2^L on the scaled points, which lie in [0, 2^L sqrt(rho)]^d; the butterfly is
run on those (unit leaves, w^A w^B = N').
"""
from __future__ import annotations

import math
from itertools import product

import numpy as np


def cis(phi):
    """exp(2 pi i phi) with phi first reduced to [0, 1)."""
    phi = np.asarray(phi, dtype=np.float64)
    return np.exp(2j * np.pi * (phi - np.floor(phi)))


def levels_for(N: float) -> int:
    """L = log2 N for N = 2^L; L = ceil(log2 N) otherwise (0 for N <= 1)."""
    if N <= 1.0:
        return 0
    return int(math.ceil(math.log2(N) - 1e-12))


def power_of_two_form(x, k, N):
    """(x', k', N') with N' = 2^L and x'.k'/N' = x.k/N: the points scaled by sqrt(N'/N)
    (unchanged when N is a power of two)."""
    L = levels_for(float(N))
    Np = 2.0 ** L
    if Np == float(N):
        return x, k, Np
    s = math.sqrt(Np / float(N))
    return x * s, k * s, Np


class Tree:
    """Step 1: the quadtree (octree) of a point set, non-empty boxes only."""

    def __init__(self, pts: np.ndarray, N: float, L: int):
        self.dim = pts.shape[1]
        self.N = float(N)
        self.L = L
        self.width = [self.N / 2 ** s for s in range(L + 1)]
        n_side = 2 ** L
        leaf = np.floor(pts / self.width[L]).astype(np.int64)
        leaf = np.clip(leaf, 0, n_side - 1)
        # boxes[s]: [n_s, dim] integer box indices at level s (sorted, unique)
        self.boxes = [None] * (L + 1)
        self.point_box = None          # leaf-box number of every point
        self.parent = [None] * (L + 1)   # parent[s][i] = box number at level s-1
        self.children = [None] * (L + 1)  # children[s][i][slot] = box number at s+1 or -1
        ub, inv = np.unique(leaf, axis=0, return_inverse=True)
        self.boxes[L] = ub.reshape(-1, self.dim)
        self.point_box = inv.reshape(-1)
        for s in range(L, 0, -1):
            par_idx = self.boxes[s] // 2
            up, pinv = np.unique(par_idx, axis=0, return_inverse=True)
            self.boxes[s - 1] = up.reshape(-1, self.dim)
            self.parent[s] = pinv.reshape(-1)
        nslot = 2 ** self.dim
        for s in range(L):
            ch = -np.ones((self.boxes[s].shape[0], nslot), dtype=np.int64)
            for i, par in enumerate(self.parent[s + 1]):
                bits = self.boxes[s + 1][i] - 2 * self.boxes[s][par]
                slot = int(sum(int(b) << (self.dim - 1 - d) for d, b in enumerate(bits)))
                ch[par, slot] = i
            self.children[s] = ch

    def corner(self, s: int) -> np.ndarray:
        return self.boxes[s] * self.width[s]

    def grid_1d(self, s: int, p: int) -> np.ndarray:
        """[n_s, dim, p]: coordinate c_d + l w_s/(p-1) of the Cartesian grid of every box."""
        q = p - 1
        return self.corner(s)[:, :, None] + (np.arange(p) * (self.width[s] / q))[None, None, :]


def _grid_points(g1: np.ndarray) -> np.ndarray:
    """[n, dim, p] per-axis coordinates -> [n, p^d, dim] grid points, l_1 slowest."""
    n, dim, p = g1.shape
    pts = np.empty((n, p ** dim, dim))
    for li, l in enumerate(product(range(p), repeat=dim)):
        for d in range(dim):
            pts[:, li, d] = g1[:, d, l[d]]
    return pts


def _axis_matrices(xg: np.ndarray, kg: np.ndarray, N: float) -> list:
    """Per axis d: (X_d)_{l l'} = exp(2 pi i xg_d[l] kg_d[l'] / N); xg, kg [n, dim, p]."""
    return [cis(xg[:, d, :, None] * kg[:, d, None, :] / N) for d in range(xg.shape[1])]


def _dense_matrix(xg: np.ndarray, kg: np.ndarray, N: float) -> np.ndarray:
    """Full p^d x p^d matrix exp(2 pi i x_l . k_l' / N) from the d-dim grid points."""
    xp = _grid_points(xg)
    kp = _grid_points(kg)
    return cis(np.einsum('zld,zmd->zlm', xp, kp) / N)


def _apply_axis(mats: np.ndarray, F: np.ndarray, axis: int) -> np.ndarray:
    """(Mat along one axis) F for a stack: mats [n,p,p], F [n,p,...,p]; contracts axis+1."""
    Fm = np.moveaxis(F, axis + 1, 1)
    sh = Fm.shape
    out = np.matmul(mats, Fm.reshape(sh[0], sh[1], -1)).reshape(sh)
    return np.moveaxis(out, 1, axis + 1)


def _solve_axis(mats: np.ndarray, U: np.ndarray, axis: int) -> np.ndarray:
    Um = np.moveaxis(U, axis + 1, 1)
    sh = Um.shape
    out = np.linalg.solve(mats, Um.reshape(sh[0], sh[1], -1)).reshape(sh)
    return np.moveaxis(out, 1, axis + 1)


def _apply(xg, kg, N, F, dense):
    """E f for a stack of pairs, E built from check grid xg and charge grid kg."""
    n, dim, p = xg.shape
    if dense:
        E = _dense_matrix(xg, kg, N)
        return np.einsum('zlm,zm->zl', E, F.reshape(n, -1)).reshape(F.shape)
    for d, Ed in enumerate(_axis_matrices(xg, kg, N)):
        F = _apply_axis(Ed, F, d)
    return F


def _solve(xg, kg, N, U, dense):
    """f with M f = U, M built from check grid xg and charge grid kg (Sec. 2.1)."""
    n, dim, p = xg.shape
    if dense:
        M = _dense_matrix(xg, kg, N)
        return np.linalg.solve(M, U.reshape(n, -1, 1)).reshape(U.shape)
    for d, Md in enumerate(_axis_matrices(xg, kg, N)):
        U = _solve_axis(Md, U, d)
    return U


def _butterfly_one(x, k, f, N, p, dense, TX, TK, L, stats, charges=None):
    dim = x.shape[1]
    q = p - 1
    tile = (p,) * dim
    # Step 2: leaf charges f^{A0 B} for every leaf B of T_K; A0 = root of T_X.
    xg0 = TX.grid_1d(0, p)                         # [1, dim, p]
    x0 = _grid_points(xg0)[0]                      # [p^d, dim]
    nB = TK.boxes[L].shape[0]
    U = np.zeros((nB, p ** dim), dtype=np.complex128)
    ph = cis(x0 @ k.T / N)                         # [p^d, nk]: exp(2 pi i x^{A0}_l . k_j / N)
    for l in range(p ** dim):
        U[:, l] = np.bincount(TK.point_box, weights=(ph[l] * f).real, minlength=nB) + \
            1j * np.bincount(TK.point_box, weights=(ph[l] * f).imag, minlength=nB)
    kgL = TK.grid_1d(L, p)
    xg = np.broadcast_to(xg0, kgL.shape)
    F = _solve(xg, kgL, N, U.reshape((nB,) + tile), dense)   # [nB, p..p]
    F = F.reshape((1, nB) + tile)                  # F[iA, iB] at stage t = L
    if stats is not None:
        stats.append((L, 1, nB))
    if charges is not None:
        charges[L] = F.copy()
    # Step 3: t = L-1 .. 0, A at level L-t of T_X, B at level t of T_K.
    for t in range(L - 1, -1, -1):
        sA, sB = L - t, t
        nA, nBt = TX.boxes[sA].shape[0], TK.boxes[sB].shape[0]
        xgA = TX.grid_1d(sA, p)                    # check grids of A
        kgB = TK.grid_1d(sB, p)                    # charge grids of B
        kgC = TK.grid_1d(sB + 1, p)                # charge grids of the children Bc
        parA = TX.parent[sA]                       # A -> A' at level sA-1
        chB = TK.children[sB]                      # B -> Bc at level sB+1 (or -1)
        iA, iB = np.meshgrid(np.arange(nA), np.arange(nBt), indexing='ij')
        iA, iB = iA.ravel(), iB.ravel()
        Ucheck = np.zeros((iA.size,) + tile, dtype=np.complex128)
        for slot in range(chB.shape[1]):
            c = chB[iB, slot]
            have = c >= 0
            if not np.any(have):
                continue
            za, zc = iA[have], c[have]
            Fc = F[parA[za], zc]                   # f^{A' Bc}
            Ucheck[have] += _apply(xgA[za], kgC[zc], N, Fc, dense)
        Fn = _solve(xgA[iA], kgB[iB], N, Ucheck, dense)
        F = Fn.reshape((nA, nBt) + tile)
        if stats is not None:
            stats.append((t, nA, nBt))
        if charges is not None:
            charges[t] = F.copy()
    # Step 4: targets of every leaf A of T_X from f^{A B0}.
    kg0 = TK.grid_1d(0, p)
    k0 = _grid_points(kg0)[0]                      # k^{B0}_l = l N/(p-1)
    FA = F[:, 0].reshape(F.shape[0], -1)           # [n leaves of T_X, p^d]
    ph = cis(x @ k0.T / N)                         # [nx, p^d]
    return np.einsum('il,il->i', ph, FA[TX.point_box])


def butterfly(x, k, f, N, p, dense: bool = False, stats: list | None = None):
    """u = butterfly approximation of eq. 1.1; f [nk] or [nrhs, nk]; returns complex128.

    `stats`, when a list, receives (t, number of A boxes, number of B boxes) per stage.
    """
    x = np.asarray(x, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    if p < 3:
        raise ValueError("p >= 3: for p = 2 the matching matrix is singular")
    x, k, N = power_of_two_form(x, k, float(N))
    L = levels_for(N)
    TX = Tree(x, N, L)
    TK = Tree(k, N, L)
    f = np.asarray(f, dtype=np.complex128)
    if f.ndim == 1:
        return _butterfly_one(x, k, f, N, p, dense, TX, TK, L, stats)
    return np.stack([_butterfly_one(x, k, fr, N, p, dense, TX, TK, L, stats if r == 0 else None)
                     for r, fr in enumerate(f)])


def stage_charges(x, k, f, N, p, dense: bool = False):
    """The equivalent charges of every stage (Sec. 2.2 steps 2 and 3) for one right-hand
    side: returns (TX, TK, L, {t: F_t}), F_t[iA, iB] the p^d tile f^{AB} of A = box iA of
    TX.boxes[L - t] and B = box iB of TK.boxes[t] (the trees of the scaled points), the
    tile's axis d the grid index along axis d."""
    x = np.asarray(x, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    x, k, N = power_of_two_form(x, k, float(N))
    L = levels_for(N)
    TX, TK = Tree(x, N, L), Tree(k, N, L)
    charges = {}
    _butterfly_one(x, k, np.asarray(f, dtype=np.complex128), N, p, dense, TX, TK, L, None, charges)
    return TX, TK, L, charges


def butterfly_matrix(x, k, N, p, dense: bool = False):
    """The butterfly as an explicit |I| x |J| matrix, one column per unit source."""
    nk = k.shape[0]
    eye = np.eye(nk, dtype=np.complex128)
    return butterfly(x, k, eye, N, p, dense).T


def pair_counts(x, k, N):
    """Stage t -> (non-empty T_X boxes at level L-t) x (non-empty T_K boxes at level t)."""
    x, k, N = power_of_two_form(np.asarray(x, float), np.asarray(k, float), float(N))
    L = levels_for(N)
    TX, TK = Tree(x, N, L), Tree(k, N, L)
    return {t: (TX.boxes[L - t].shape[0], TK.boxes[t].shape[0]) for t in range(L + 1)}
