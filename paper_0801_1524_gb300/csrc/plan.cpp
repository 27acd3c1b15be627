// Host plan: trees (Sec. 2.2 step 1), transfer operators (eqs. M1, E1), work chunks.
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace bfly {

namespace {

inline uint64_t morton(const int64_t *a, int dim, int L) {
  uint64_t key = 0;
  for (int b = L - 1; b >= 0; --b)
    for (int d = 0; d < dim; ++d) key = (key << 1) | (uint64_t)((a[d] >> b) & 1);
  return key;
}

// sin(pi * num / den) and cos(pi * num / den) for an exact rational angle.
inline double sinpi_rat(double num, double den) { return std::sin(M_PI * (num / den)); }

}  // namespace

std::string build_tree(HostTree &T, int dim, int L, int64_t n, const double *pts) {
  T = HostTree();
  T.dim = dim;
  T.L = L;
  T.n = n;
  const int64_t side = int64_t(1) << L;
  std::vector<int64_t> leaf((size_t)(n * dim));
  std::vector<double> off((size_t)(n * dim));
  std::vector<uint64_t> key((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    for (int d = 0; d < dim; ++d) {
      const double v = pts[i * dim + d];
      if (!(v >= 0.0) || !(v <= (double)side)) return "point coordinate outside [0, N]";
      int64_t a = (int64_t)std::floor(v);
      if (a > side - 1) a = side - 1;  // the far edge N belongs to the last box
      leaf[i * dim + d] = a;
      off[i * dim + d] = v - (double)a;  // exact: v and a differ by less than 2
    }
    key[i] = morton(&leaf[i * dim], dim, L);
  }
  T.perm.resize((size_t)n);
  std::iota(T.perm.begin(), T.perm.end(), 0);
  std::stable_sort(T.perm.begin(), T.perm.end(),
                   [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  T.off.resize((size_t)(n * dim));
  T.point_leaf.resize((size_t)n);
  T.idx.assign(L + 1, {});
  T.cs.assign(L + 1, {});
  // leaves: runs of equal keys in sorted order
  std::vector<uint64_t> lkey;
  for (int64_t s = 0; s < n; ++s) {
    const int32_t i = T.perm[s];
    for (int d = 0; d < dim; ++d) T.off[s * dim + d] = off[i * dim + d];
    if (s == 0 || key[i] != lkey.back()) {
      lkey.push_back(key[i]);
      T.leaf_start.push_back((int32_t)s);
      for (int d = 0; d < dim; ++d) T.idx[L].push_back((int32_t)leaf[i * dim + d]);
    }
    T.point_leaf[s] = (int32_t)lkey.size() - 1;
  }
  T.leaf_start.push_back((int32_t)n);
  // coarser levels: parents are runs of equal key >> dim
  for (int s = L - 1; s >= 0; --s) {
    std::vector<uint64_t> pkey;
    const int64_t nc = (int64_t)lkey.size();
    for (int64_t c = 0; c < nc; ++c) {
      const uint64_t pk = lkey[c] >> dim;
      if (c == 0 || pk != pkey.back()) {
        pkey.push_back(pk);
        T.cs[s].push_back((int32_t)c);
        for (int d = 0; d < dim; ++d) T.idx[s].push_back(T.idx[s + 1][c * dim + d] >> 1);
      }
    }
    T.cs[s].push_back((int32_t)nc);
    lkey.swap(pkey);
  }
  return "";
}

void leaf_weights(int p, double tau, double *w) {
  // G_{ll'} = exp(2 pi i l l'/q^2) is the Vandermonde matrix of the nodes
  // z_m = exp(2 pi i m/q^2) and v(tau)_l = z(tau)^l with z(tau) = exp(2 pi i tau/q), so
  // G^{-1} v(tau) holds the Lagrange basis polynomials of those nodes at z(tau).  As
  // z - z_n = 2i sin((theta - phi_n)/2) e^{i(theta + phi_n)/2}, the product form is
  //   w_m = e^{i pi (tau - m/q)} prod_{n != m} sin(pi (tau - n/q)/q) / sin(pi (m-n)/q^2),
  // which needs no inverse of the ill-conditioned G.
  const int q = p - 1;
  for (int m = 0; m < p; ++m) {
    double num = 1.0, den = 1.0;
    for (int n = 0; n < p; ++n) {
      if (n == m) continue;
      num *= std::sin(M_PI * (tau - (double)n / q) / q);
      den *= sinpi_rat((double)(m - n), (double)q * q);
    }
    const double ang = M_PI * (tau - (double)m / q);
    w[2 * m] = std::cos(ang) * num / den;
    w[2 * m + 1] = std::sin(ang) * num / den;
  }
}

std::vector<double> transfer_table(int p, bool adjoint) {
  // For A at level s with index a, w^A w^B = N, parent charges on the grid of B and
  // child charges on the grid of Bc (child offset bit delta), the matching condition of
  // Sec. 2.1 with the evaluation of Fig. 1 gives, per axis, f^{AB} = T f^{A'Bc} with
  //   T_{m l} = omega^{-a m} e^{2 pi i a tau_l} w_m(tau_l),  tau_l = (delta + l/q)/2,
  // omega = e^{2 pi i/q}: the Lagrange weights of the child grid point tau_l on the
  // parent grid, times the box phases of eqs. M1 and E1 (the index of B cancels).  T
  // depends on a only through alpha = a mod 2q.
  const int q = p - 1;
  const int nops = 4 * q;
  std::vector<double> T((size_t)nops * p * p * 2, 0.0);
  std::vector<double> w((size_t)2 * p);
  for (int alpha = 0; alpha < 2 * q; ++alpha) {
    for (int delta = 0; delta < 2; ++delta) {
      const int op = alpha * 2 + delta;
      for (int l = 0; l < p; ++l) {
        const double tau = (double)(delta * q + l) / (2.0 * q);
        leaf_weights(p, tau, w.data());
        // e^{2 pi i alpha tau} = e^{i pi (alpha (delta q + l) mod 2q)/q}
        const int n1 = (alpha * (delta * q + l)) % (2 * q);
        for (int m = 0; m < p; ++m) {
          // omega^{-alpha m} = e^{-i pi 2 (alpha m mod q)/q}
          const int n2 = (2 * ((alpha * m) % q)) % (2 * q);
          const int nn = ((n1 - n2) % (2 * q) + 2 * q) % (2 * q);
          const double c = std::cos(M_PI * nn / q), s = std::sin(M_PI * nn / q);
          const double wr = w[2 * m], wi = w[2 * m + 1];
          const double re = c * wr - s * wi, im = c * wi + s * wr;
          const size_t at = adjoint ? (((size_t)op * p + l) * p + m) : (((size_t)op * p + m) * p + l);
          T[2 * at] = re;
          T[2 * at + 1] = adjoint ? -im : im;
        }
      }
    }
  }
  return T;
}

std::vector<Chunk> make_chunks(const std::vector<int32_t> &csAp, const std::vector<int32_t> &csB,
                               bool adjoint, int tile_cap) {
  std::vector<Chunk> out;
  const int64_t nAp = (int64_t)csAp.size() - 1, nB = (int64_t)csB.size() - 1;
  const int64_t units = nAp * nB;
  Chunk cur{0, 0, 0, INT16_MAX};
  int tiles = 0, ins = 0, outs = 0;
  auto flush = [&]() {
    if (cur.nu > 0) out.push_back(cur);
    cur = Chunk{0, 0, 0, INT16_MAX};
    tiles = ins = outs = 0;
  };
  for (int64_t u = 0; u < units; ++u) {
    const int64_t iAp = u / nB, iB = u % nB;
    const int na = csAp[iAp + 1] - csAp[iAp];
    const int nc = csB[iB + 1] - csB[iB];
    const int nin = adjoint ? na : nc;
    const int nout = adjoint ? nc : na;
    const int need = nin + nout * nin;
    if (need > tile_cap || nout > kMaxOut || nin > kMaxIn) {
      // a unit larger than one block: split its outputs
      flush();
      const int g = std::max(1, std::min(kMaxOut, (tile_cap - nin) / nin));
      for (int o = 0; o < nout; o += g)
        out.push_back(Chunk{u, 1, (int16_t)o, (int16_t)std::min(nout, o + g)});
      continue;
    }
    if (cur.nu > 0 && (tiles + need > tile_cap || ins + nin > kMaxIn || outs + nout > kMaxOut ||
                       cur.nu + 1 > kMaxUnits))
      flush();
    if (cur.nu == 0) cur.u0 = u;
    cur.nu += 1;
    tiles += need;
    ins += nin;
    outs += nout;
  }
  flush();
  return out;
}

}  // namespace bfly
