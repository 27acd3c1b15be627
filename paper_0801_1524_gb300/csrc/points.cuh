// Steps 2 and 4 of Sec. 2.2 and their adjoints, and the per-point weights they use.
//
// Leaf step (step 2): for every leaf B of T_K the equivalent charges for the root A0 of
// T_X are f^{A0 B} = sum_{j in B} f_j (x)_d w(tau_{j,d}), tau = k_j / rho - b the offset of
// the source in its leaf (rho = N / 2^L wide) and w(tau) = G^{-1} v(tau) (eq. M1 with
// c^{A0} = 0).
// Final step (step 4): u_i = sum_l prod_d e^{2 pi i rho l_d sigma_{i,d}/q} g^{A B0}_l, with
// sigma = x_i / rho - a the offset of x_i in its leaf a (k^{B0}_l = l N/q) and g the
// rescaled charges g_l = e^{2 pi i rho a l/q} f_l of the recursive step, which absorb
// the leaf's own phase.
// Both are "spread" (points -> one tile per leaf) or "interp" (one tile per leaf ->
// points) with per-point weights W[point][d][l]; the adjoint sweep uses the other of
// the two with conj(W).
#pragma once

#include "common.cuh"

namespace bfly {

// tile[b][l] = sum_{j in leaf b} val_j prod_d W_j[d][l_d]   (conj(W) when a.conj)
template <typename R, int D, int P>
__global__ void __launch_bounds__(256) spread_kernel(const PointArgs a) {
  using C = typename Cx<R>::T;
  constexpr int PD = ipow(P, D);
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (w >= a.nbox * PD) return;
  const int64_t b = w / PD;
  const int l = (int)(w - b * PD);
  int ld[D];
  {
    int rem = l;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) {
      ld[d] = rem % P;
      rem /= P;
    }
  }
  const C *W = reinterpret_cast<const C *>(a.W);
  C acc = cmk((R)0, (R)0);
  const int j0 = a.leaf_start[b], j1 = a.leaf_start[b + 1];
  for (int j = j0; j < j1; ++j) {
    const C v = load_io<C>(a.vin, (int64_t)r * a.n_total + a.perm[j], a.io64);
    C wt = W[((size_t)j * D + 0) * P + ld[0]];
#pragma unroll
    for (int d = 1; d < D; ++d) wt = cmul(wt, W[((size_t)j * D + d) * P + ld[d]]);
    acc = a.conj ? cfma_conj(wt, v, acc) : cfma(wt, v, acc);
  }
  reinterpret_cast<C *>(a.vout)[(size_t)r * a.tile_rhs + (size_t)b * a.tile_stride + l] = acc;
}

// val_i = sum_l prod_d W_i[d][l_d] tile[leaf(i)][l]   (conj(W) when a.conj)
template <typename R, int D, int P>
__global__ void __launch_bounds__(256) interp_kernel(const PointArgs a) {
  using C = typename Cx<R>::T;
  constexpr int PD = ipow(P, D);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= a.n_total) return;
  const C *W = reinterpret_cast<const C *>(a.W) + (size_t)i * D * P;
  C w[D][P];
#pragma unroll
  for (int d = 0; d < D; ++d)
#pragma unroll
    for (int l = 0; l < P; ++l) w[d][l] = a.conj ? cconj(W[d * P + l]) : W[d * P + l];
  const C *tile = reinterpret_cast<const C *>(a.vin) + (size_t)r * a.tile_rhs +
                  (size_t)a.point_leaf[i] * a.tile_stride;
  C acc = cmk((R)0, (R)0);
  if (D == 2) {
#pragma unroll
    for (int l0 = 0; l0 < P; ++l0) {
      C s = cmk((R)0, (R)0);
#pragma unroll
      for (int l1 = 0; l1 < P; ++l1) s = cfma(w[D - 1][l1], tile[l0 * P + l1], s);
      acc = cfma(w[0][l0], s, acc);
    }
  } else {
#pragma unroll
    for (int l0 = 0; l0 < P; ++l0) {
      C s1 = cmk((R)0, (R)0);
      for (int l1 = 0; l1 < P; ++l1) {
        C s2 = cmk((R)0, (R)0);
#pragma unroll
        for (int l2 = 0; l2 < P; ++l2) s2 = cfma(w[D - 1][l2], tile[(l0 * P + l1) * P + l2], s2);
        s1 = cfma(w[D > 2 ? 1 : 0][l1], s2, s1);
      }
      acc = cfma(w[0][l0], s1, acc);
    }
  }
  store_io(a.vout, (int64_t)r * a.n_total + a.perm[i], acc, a.io64);
}

// Plan-time weights, computed in FP64 and stored in the plan's precision R; tau is the
// offset of the point from its leaf corner in leaf widths, rho = N / 2^L the leaf width.
//   kind 0 (T_K, step 2): W[j][d][m] = w_m(tau_{j,d}) by the Lagrange product form
//          e^{i pi rho (tau - m/q)} prod_{n != m} sin(pi rho (tau - n/q)/q) * inv_den[m];
//   kind 1 (T_X, step 4): W[i][d][l] = exp(2 pi i rho l tau_{i,d}/q).
constexpr int kMaxP = 9;
template <typename R>
__global__ void weights_kernel(int64_t n, int dim, int p, double rho, int kind, const double *off,
                               const double *inv_den, typename Cx<R>::T *W) {
  using C = typename Cx<R>::T;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * dim) return;
  const int q = p - 1;
  const double tau = off[t];
  C *out = W + (size_t)t * p;
  if (kind == 0) {
    double s[kMaxP], pre[kMaxP + 1], suf[kMaxP + 1];
    for (int n2 = 0; n2 < p; ++n2) s[n2] = sinpi(rho * (tau - (double)n2 / q) / q);
    pre[0] = 1.0;
    for (int n2 = 0; n2 < p; ++n2) pre[n2 + 1] = pre[n2] * s[n2];
    suf[p] = 1.0;
    for (int n2 = p - 1; n2 >= 0; --n2) suf[n2] = suf[n2 + 1] * s[n2];
    for (int m = 0; m < p; ++m) {
      const double mag = pre[m] * suf[m + 1] * inv_den[m];
      double sn, cs;
      sincospi(rho * (tau - (double)m / q), &sn, &cs);
      out[m] = cmk((R)(cs * mag), (R)(sn * mag));
    }
  } else {
    for (int l = 0; l < p; ++l) {
      double sn, cs;
      sincospi(2.0 * rho * (double)l * tau / q, &sn, &cs);
      out[l] = cmk((R)cs, (R)sn);
    }
  }
}

}  // namespace bfly
