// Steps 2 and 4 of Sec. 2.2 and their adjoints, and the per-point weights they use.
//
// Leaf step (step 2): for every leaf B of T_K the equivalent charges for the root A0 of
// T_X are f^{A0 B} = sum_{j in B} f_j (x)_d w(tau_{j,d}), tau = k_j - b the offset of the
// source in its unit leaf and w(tau) = G^{-1} v(tau) (eq. M1 with c^{A0} = 0).
// Final step (step 4): u_i = sum_l prod_d e^{2 pi i l_d sigma_{i,d}/q} g^{A B0}_l, with
// sigma = x_i - a the offset of x_i in its unit leaf a (k^{B0}_l = l N/q) and g the
// rescaled charges g_l = e^{2 pi i a l/q} f_l of the recursive step, which absorb the
// leaf's own phase.  (Points are the scaled ones: N = 2^L here.)
// Both are "spread" (points -> one tile per leaf) or "interp" (one tile per leaf ->
// points) with per-point weights W[point][d][l]; the adjoint sweep uses the other of
// the two with conj(W).
#pragma once

#include "common.cuh"

namespace bfly {

constexpr int kPointThreads = 256;
constexpr int kSpreadPerThread = 4;  // tile elements per thread

// tile[b][l] = sum_{j in leaf b} val_j prod_d W_j[d][l_d]   (conj(W) when a.conj)
// A block covers 1024 consecutive tile elements (b, l) (four per thread, 256 apart so that
// the stores are coalesced), i.e. the consecutive leaves of those elements, whose points
// are consecutive in sorted order.  The block stages those points (value gathered through
// perm, weight rows) in shared memory, a batch at a time, so that every point is read
// from memory once and the loads of a batch are in flight together; then each thread sums
// the batch's points of its elements' leaves.
constexpr int kPointRhs = 4;  // right-hand sides per block (leaf step) or lane group (final step)

template <typename R, int D, int P>
__global__ void __launch_bounds__(kPointThreads, 4) spread_kernel(const PointArgs a) {
  using C = typename Cx<R>::T;
  constexpr int PD = ipow(P, D), E = kPointThreads * kSpreadPerThread;
  constexpr int BATCH = (24576 / ((D * P + 1) * (int)sizeof(C))) / 32 * 32;
  __shared__ C s_v[BATCH];
  __shared__ C s_w[BATCH][D * P];
  const int64_t n_el = a.nbox * PD;
  const int64_t e0 = (int64_t)blockIdx.x * E;
  // right-hand sides r0 .. r0 + nb - 1 of this block: the weights, leaf ranges and
  // permutation are read once for all of them
  const int r0 = blockIdx.y * kPointRhs, nb = min(kPointRhs, a.nrhs - r0);
  // element k of this thread: tile element l (< PD) of leaf bk (the plan's leaves number
  // fewer than 2^31), its points j0 .. j1 - 1 in sorted order
  // (the leaf's point range is read where it is used, an L1 hit, so that fewer values stay
  // live across the right-hand sides)
  int bk[kSpreadPerThread], lt[kSpreadPerThread];
#pragma unroll
  for (int k = 0; k < kSpreadPerThread; ++k) {
    const int64_t w = e0 + threadIdx.x + k * kPointThreads;
    const bool on = w < n_el;
    bk[k] = on ? (int)(w / PD) : -1;
    lt[k] = on ? (int)(w - (int64_t)bk[k] * PD) : 0;
  }
  pdl_trigger();
  // the block's points: those of leaves e0/PD .. (last element)/PD.  The leaf ranges, the
  // permutation and the weights are plan data, read before the dependency wait; only the
  // point values (the caller's) and the output tiles (read by the predecessor's sweep)
  // wait for the predecessor grid.
  const int64_t e1 = min(n_el, e0 + E);
  const int jb0 = a.leaf_start[e0 / PD], jb1 = a.leaf_start[(e1 - 1) / PD + 1];
  const C *W = reinterpret_cast<const C *>(a.W);
  constexpr int PJ = (BATCH + kPointThreads - 1) / kPointThreads;
  bool waited = false;
  C acc[kSpreadPerThread];
  int pj[PJ];
  // stages the weights and permutation entries of points pb .. pb + n - 1
  auto stage_plan = [&](int pb, int n) {
#pragma unroll
    for (int q = 0; q < PJ; ++q) {
      const int t = threadIdx.x + q * kPointThreads;
      pj[q] = t < n ? a.perm[pb + t] : 0;
    }
    for (int t = threadIdx.x; t < n * D * P; t += kPointThreads) {
      const C wv = W[(size_t)pb * D * P + t];
      s_w[t / (D * P)][t % (D * P)] = a.conj ? cconj(wv) : wv;
    }
  };
  // gathers the values of right-hand side r of points pb .., then (after a barrier) adds
  // their terms to the accumulators
  auto accumulate = [&](int pb, int n, int r) {
#pragma unroll
    for (int q = 0; q < PJ; ++q) {
      const int t = threadIdx.x + q * kPointThreads;
      if (t < n) s_v[t] = load_io<C>(a.vin, (int64_t)r * a.n_total + pj[q], a.io64);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSpreadPerThread; ++k) {
      if (bk[k] < 0) continue;
      const int ja = max(a.leaf_start[bk[k]], pb) - pb, jz = min(a.leaf_start[bk[k] + 1], pb + n) - pb;
      // the index of element l along each axis (axis 0 slowest)
      int ld[D];
      int rem = lt[k];
#pragma unroll
      for (int d = D - 1; d >= 0; --d) {
        ld[d] = rem % P;
        rem /= P;
      }
      for (int j = ja; j < jz; ++j) {
        C wt = s_w[j][ld[0]];
#pragma unroll
        for (int d = 1; d < D; ++d) wt = cmul(wt, s_w[j][d * P + ld[d]]);
        acc[k] = cfma(wt, s_v[j], acc[k]);
      }
    }
    __syncthreads();
  };
  auto store = [&](int r) {
#pragma unroll
    for (int k = 0; k < kSpreadPerThread; ++k)
      if (bk[k] >= 0)
        reinterpret_cast<C *>(a.vout)[(size_t)r * a.tile_rhs + (size_t)bk[k] * a.tile_stride + lt[k]] = acc[k];
  };
  if (jb1 - jb0 <= BATCH) {
    // the usual case: the block's points fit one batch, staged once for every right-hand side
    stage_plan(jb0, jb1 - jb0);
    pdl_wait();
    for (int q = 0; q < nb; ++q) {
#pragma unroll
      for (int k = 0; k < kSpreadPerThread; ++k) acc[k] = cmk((R)0, (R)0);
      accumulate(jb0, jb1 - jb0, r0 + q);
      store(r0 + q);
    }
    return;
  }
  for (int q = 0; q < nb; ++q) {
#pragma unroll
    for (int k = 0; k < kSpreadPerThread; ++k) acc[k] = cmk((R)0, (R)0);
    for (int pb = jb0; pb < jb1; pb += BATCH) {
      const int n = min(BATCH, jb1 - pb);
      stage_plan(pb, n);
      if (!waited) {
        pdl_wait();
        waited = true;
      }
      accumulate(pb, n, r0 + q);
    }
    if (!waited) {
      pdl_wait();
      waited = true;
    }
    store(r0 + q);
  }
}

constexpr int kInterpLanes = 8;  // lanes per target

// val_i = sum_l prod_d W_i[d][l_d] tile[leaf(i)][l]   (conj(W) when a.conj)
// Eight lanes per target: lane g sums the slices l_0 = g and g + 8 of the tile
// (sum over l_1.. first, then the weight of l_0), and the eight partial sums are added
// with shuffles; lane 0 writes the result in caller order.  A lane group takes up to
// kPointRhs right-hand sides of its target one after the other, reading the target's
// weights, leaf and caller index once.
template <typename R, int D, int P>
__global__ void __launch_bounds__(kPointThreads) interp_kernel(const PointArgs a) {
  using C = typename Cx<R>::T;
  const int64_t gt = (int64_t)blockIdx.x * kPointThreads + threadIdx.x;
  const int64_t i = gt / kInterpLanes;
  const int g = (int)(gt % kInterpLanes);
  const int r0 = blockIdx.y * kPointRhs, nb = min(kPointRhs, a.nrhs - r0);
  const bool active = i < a.n_total;
  // the plan's weights and leaf indices are read before the predecessor grid has ended;
  // the tiles it writes after
  pdl_trigger();
  const C *Wi = reinterpret_cast<const C *>(a.W) + (size_t)(active ? i : 0) * D * P;
  const C *tile0 = reinterpret_cast<const C *>(a.vin) + (size_t)(active ? a.point_leaf[i] : 0) * a.tile_stride;
  C wl[P];  // weights of the last axis
#pragma unroll
  for (int l = 0; l < P; ++l)
    wl[l] = !active ? cmk((R)0, (R)0) : a.conj ? cconj(Wi[(D - 1) * P + l]) : Wi[(D - 1) * P + l];
  pdl_wait();
  for (int q = 0; q < nb; ++q) {
    const int r = r0 + q;
    const C *tile = tile0 + (size_t)r * a.tile_rhs;
    C acc = cmk((R)0, (R)0);
    if (active) {
#pragma unroll
      for (int h = 0; h < (P + kInterpLanes - 1) / kInterpLanes; ++h) {
        const int l0 = g + h * kInterpLanes;
        if (l0 >= P) break;
        C s1 = cmk((R)0, (R)0);
        if (D == 2) {
#pragma unroll
          for (int l1 = 0; l1 < P; ++l1) s1 = cfma(wl[l1], tile[l0 * P + l1], s1);
        } else {
#pragma unroll 1
          for (int l1 = 0; l1 < P; ++l1) {
            C s2 = cmk((R)0, (R)0);
#pragma unroll
            for (int l2 = 0; l2 < P; ++l2) s2 = cfma(wl[l2], tile[(l0 * P + l1) * P + l2], s2);
            const C w1 = a.conj ? cconj(Wi[P + l1]) : Wi[P + l1];
            s1 = cfma(w1, s2, s1);
          }
        }
        const C w0 = a.conj ? cconj(Wi[l0]) : Wi[l0];
        acc = cfma(w0, s1, acc);
      }
    }
#pragma unroll
    for (int o = kInterpLanes / 2; o > 0; o /= 2) acc = cadd(acc, shfl_xor_c(acc, o));
    if (active && g == 0) store_io(a.vout, (int64_t)r * a.n_total + a.perm[i], acc, a.io64);
  }
}

// Plan-time weights, computed in FP64 and stored in the plan's precision R; tau is the
// offset of the (scaled) point from its leaf corner.
//   kind 0 (T_K, step 2): W[j][d][m] = w_m(tau_{j,d}) by the Lagrange product form
//          e^{i pi (tau - m/q)} prod_{n != m} sin(pi (tau - n/q)/q) * inv_den[m];
//   kind 1 (T_X, step 4): W[i][d][l] = exp(2 pi i l tau_{i,d}/q).
constexpr int kMaxP = 9;
template <typename R>
__global__ void weights_kernel(int64_t n, int dim, int p, int kind, const double *off,
                               const double *inv_den, typename Cx<R>::T *W) {
  using C = typename Cx<R>::T;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * dim) return;
  const int q = p - 1;
  const double tau = off[t];
  C *out = W + (size_t)t * p;
  if (kind == 0) {
    double s[kMaxP], pre[kMaxP + 1], suf[kMaxP + 1];
    for (int n2 = 0; n2 < p; ++n2) s[n2] = sinpi((tau - (double)n2 / q) / q);
    pre[0] = 1.0;
    for (int n2 = 0; n2 < p; ++n2) pre[n2 + 1] = pre[n2] * s[n2];
    suf[p] = 1.0;
    for (int n2 = p - 1; n2 >= 0; --n2) suf[n2] = suf[n2 + 1] * s[n2];
    for (int m = 0; m < p; ++m) {
      const double mag = pre[m] * suf[m + 1] * inv_den[m];
      double sn, cs;
      sincospi(tau - (double)m / q, &sn, &cs);
      out[m] = cmk((R)(cs * mag), (R)(sn * mag));
    }
  } else {
    for (int l = 0; l < p; ++l) {
      double sn, cs;
      sincospi(2.0 * (double)l * tau / q, &sn, &cs);
      out[l] = cmk((R)cs, (R)sn);
    }
  }
}

}  // namespace bfly
