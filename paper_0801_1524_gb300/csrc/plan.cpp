// Host plan: trees (Sec. 2.2 step 1), transfer operators (eqs. M1, E1), work chunks.
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

namespace bfly {

namespace {

inline uint64_t morton(const int64_t *a, int dim, int L) {
  uint64_t key = 0;
  for (int b = L - 1; b >= 0; --b)
    for (int d = 0; d < dim; ++d) key = (key << 1) | (uint64_t)((a[d] >> b) & 1);
  return key;
}


}  // namespace

std::string build_tree(HostTree &T, int dim, int L, double N, double scale, int64_t n, const double *pts) {
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
      if (!(v >= 0.0) || !(v <= N)) return "point coordinate outside [0, N]";
      const double u = scale == 1.0 ? v : v * scale;  // in [0, 2^L]
      int64_t a = (int64_t)std::floor(u);
      if (a > side - 1) a = side - 1;  // the far edge belongs to the last box
      leaf[i * dim + d] = a;
      off[i * dim + d] = u - (double)a;  // exact: u and a differ by less than 2
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
      den *= std::sin(M_PI * ((double)(m - n) / ((double)q * q)));
    }
    const double ang = M_PI * (tau - (double)m / q);
    w[2 * m] = std::cos(ang) * num / den;
    w[2 * m + 1] = std::sin(ang) * num / den;
  }
}

void transfer_factors(int p, bool adjoint, double *W, double *phi) {
  // C^{(gamma,delta)} = W(delta) diag(phi_gamma), W(delta)_{ml} = w_m(tau_l),
  // phi_0 = 1, phi_1[l] = e^{2 pi i tau_l} = e^{i pi (delta q + l)/q}; the adjoint
  // operator is diag(conj phi_gamma) W(delta)^H.
  const int q = p - 1;
  std::vector<double> w((size_t)2 * p);
  for (int delta = 0; delta < 2; ++delta)
    for (int l = 0; l < p; ++l) {
      const double tau = (double)(delta * q + l) / (2.0 * q);
      leaf_weights(p, tau, w.data());
      for (int m = 0; m < p; ++m) {
        const size_t at = adjoint ? (((size_t)delta * p + l) * p + m) : (((size_t)delta * p + m) * p + l);
        W[2 * at] = w[2 * m];
        W[2 * at + 1] = adjoint ? -w[2 * m + 1] : w[2 * m + 1];
      }
      const double ang = M_PI * (double)(delta * q + l) / q;
      phi[2 * (delta * p + l)] = std::cos(ang);
      phi[2 * (delta * p + l) + 1] = adjoint ? -std::sin(ang) : std::sin(ang);
    }
}

namespace {

// Per-unit program before slot numbering: tiles of every pass keyed by a D-bit mask whose
// bits 0..k come from the output side and bits k+1..D-1 from the input side.
struct UnitProg {
  int n_in = 0;
  int in_key[8];
  int32_t in_tile[8];
  int n_pass[3] = {0, 0, 0};
  int key[3][8];
  // sources: index into the previous pass (or inputs) of this unit, -1 if absent
  int src[3][8][2];
  int op[3][8][2];
  int32_t out_tile[8];
};

// The unit (A', B) = (iAp, iB) of one stage (trees S).
UnitProg build_unit(int D, const StageTrees &S, int64_t iAp, int64_t iB, bool adjoint) {
  const std::vector<int32_t> &csAp = *S.csAp, &xidx = *S.xidx, &csB = *S.csB, &kidx = *S.kidx;
  const int64_t nB = (int64_t)csB.size() - 1, nBc = (int64_t)kidx.size() / D;
  const int64_t in_row = adjoint ? nB : nBc, out_row = adjoint ? nBc : nB;
  auto lo = [](int k) { return (1 << (k + 1)) - 1; };     // bits 0..k
  auto hi = [&](int k) { return ((1 << D) - 1) & ~lo(k); };  // bits k+1..D-1
  const int a0 = csAp[iAp], a1 = csAp[iAp + 1];
  const int c0 = csB[iB], c1 = csB[iB + 1];
  UnitProg U;
  int gam[8], ng = 0, del[8], nd = 0;
  int32_t gtile[8], dtile[8];
  for (int a = a0; a < a1; ++a) {
    int g = 0;
    for (int d = 0; d < D; ++d) g |= (xidx[(int64_t)a * D + d] & 1) << d;
    gam[ng] = g;
    gtile[ng++] = a;
  }
  for (int c = c0; c < c1; ++c) {
    int dl = 0;
    for (int d = 0; d < D; ++d) dl |= (kidx[(int64_t)c * D + d] & 1) << d;
    del[nd] = dl;
    dtile[nd++] = c;
  }
  // inputs and outputs with their keys and global tiles
  const int n_in = adjoint ? ng : nd, n_out = adjoint ? nd : ng;
  const int *ikey = adjoint ? gam : del, *okey = adjoint ? del : gam;
  U.n_in = n_in;
  for (int i = 0; i < n_in; ++i) {
    U.in_key[i] = ikey[i];
    U.in_tile[i] = adjoint ? (int32_t)((int64_t)gtile[i] * in_row + iB) : (int32_t)(iAp * in_row + dtile[i]);
  }
  for (int k = 0; k < D; ++k) {
    // needed keys of pass k: out-prefix (bits 0..k) x in-suffix (bits k+1..)
    int nk2 = 0;
    for (int o = 0; o < n_out; ++o)
      for (int i = 0; i < n_in; ++i) {
        const int K = (okey[o] & lo(k)) | (ikey[i] & hi(k));
        bool seen = false;
        for (int j = 0; j < nk2; ++j) seen |= U.key[k][j] == K;
        if (!seen) U.key[k][nk2++] = K;
      }
    U.n_pass[k] = nk2;
    for (int v = 0; v < nk2; ++v) {
      const int K = U.key[k][v];
      const int obit = (K >> k) & 1;
      for (int b = 0; b < 2; ++b) {
        const int Sk = (K & ~(1 << k)) | (b << k);
        int found = -1;
        if (k == 0) {
          for (int i = 0; i < n_in; ++i)
            if (U.in_key[i] == Sk) found = i;  // input keys are all in-side bits
        } else {
          for (int j = 0; j < U.n_pass[k - 1]; ++j)
            if (U.key[k - 1][j] == Sk) found = j;
        }
        U.src[k][v][b] = found;
        // operator gamma*2 + delta: forward, gamma is the output (A) bit and delta = b;
        // adjoint, gamma is the input (A) bit b and delta the output (Bc) bit
        U.op[k][v][b] = adjoint ? b * 2 + obit : obit * 2 + b;
      }
    }
  }
  for (int v = 0; v < U.n_pass[D - 1]; ++v) {
    // the last pass's keys are output keys: find that output's tile
    for (int o = 0; o < n_out; ++o)
      if (okey[o] == U.key[D - 1][v])
        U.out_tile[v] = adjoint ? (int32_t)(iAp * out_row + dtile[o]) : (int32_t)((int64_t)gtile[o] * out_row + iB);
  }
  return U;
}

// A unit of a step: its subunits level by level (one level: a single unit).
struct StepUnit {
  std::vector<UnitProg> lev[kMaxLevels];
};

}  // namespace

StageProgram make_step_program(int dim, int p, const StageTrees *st, int levels, bool adjoint, ChunkCaps caps,
                               bool *fits) {
  StageProgram prog;
  const int D = dim, NL = levels, NP = levels * dim;
  if (fits) *fits = true;
  // running totals of the chunk being filled: inputs and the outputs of every pass
  struct Tot {
    int in = 0, pass[kMaxPasses] = {0, 0, 0, 0, 0, 0};
  };
  auto add = [&](Tot &t, const StepUnit &m) {
    for (const UnitProg &u : m.lev[0]) t.in += u.n_in;
    for (int l = 0; l < NL; ++l)
      for (const UnitProg &u : m.lev[l])
        for (int k = 0; k < D; ++k) t.pass[l * D + k] += u.n_pass[k];
  };
  // pass j writes the scratch buffer (even j) or the input buffer (odd j); the last
  // pass's outputs are staged there and written back as runs
  auto within = [&](const Tot &t) {
    int need0 = t.in, need1 = 0, items = 0;
    for (int j = 0; j < NP; ++j) {
      if (j & 1) need0 = std::max(need0, t.pass[j]);
      else need1 = std::max(need1, t.pass[j]);
      items += t.pass[j];
    }
    const int nout = t.pass[NP - 1];
    const int meta = kBlobHeader + 8 * items + 8 * nout + 15;
    return need0 <= caps.cap0 && need1 <= caps.cap1 && nout <= caps.max_out && meta <= caps.meta_bytes;
  };

  std::vector<StepUnit> cur;
  Tot tot;
  auto flush = [&]() {
    if (cur.empty()) return;
    ChunkDesc cd{};
    std::vector<const UnitProg *> su[kMaxLevels];
    for (const StepUnit &m : cur)
      for (int l = 0; l < NL; ++l)
        for (const UnitProg &u : m.lev[l]) su[l].push_back(&u);
    // inputs of the chunk in global order: slot = rank, so that runs are contiguous
    std::vector<std::pair<int32_t, int>> order;  // (global tile, unit-local key index)
    std::vector<int> base_in(su[0].size());
    int bi = 0;
    for (size_t u = 0; u < su[0].size(); ++u) {
      base_in[u] = bi;
      for (int i = 0; i < su[0][u]->n_in; ++i) order.push_back({su[0][u]->in_tile[i], bi + i});
      bi += su[0][u]->n_in;
    }
    cd.n_in = bi;
    std::vector<std::pair<int32_t, int>> sorted = order;
    std::sort(sorted.begin(), sorted.end());
    std::vector<int> slot_of(order.size());
    for (size_t r = 0; r < sorted.size(); ++r) slot_of[sorted[r].second] = (int)r;
    prog.in_off.push_back((int32_t)prog.in_tiles.size());
    cd.run_off = (int32_t)prog.runs.size();
    for (size_t r = 0; r < sorted.size(); ++r) {
      prog.in_tiles.push_back(sorted[r].first);
      if (r > 0 && sorted[r].first == sorted[r - 1].first + 1 && prog.runs.back().count < 0xffff)
        prog.runs.back().count++;
      else
        prog.runs.push_back(Run{sorted[r].first, (uint16_t)r, 1});
    }
    cd.n_runs = (int32_t)prog.runs.size() - cd.run_off;
    // output slots of every pass, numbered subunit by subunit
    std::vector<int> base[kMaxLevels][3];
    for (int l = 0; l < NL; ++l)
      for (int k = 0; k < D; ++k) {
        base[l][k].resize(su[l].size());
        int b = 0;
        for (size_t u = 0; u < su[l].size(); ++u) {
          base[l][k][u] = b;
          b += su[l][u]->n_pass[k];
        }
      }
    // the last level's outputs: staging slots in global order, so that they form runs
    std::vector<int32_t> outs;
    for (const UnitProg *u : su[NL - 1])
      for (int v = 0; v < u->n_pass[D - 1]; ++v) outs.push_back(u->out_tile[v]);
    std::vector<int32_t> osorted = outs;
    std::sort(osorted.begin(), osorted.end());
    std::vector<std::pair<int32_t, int>> inter;  // (global tile, slot) of the previous level's outputs
    std::vector<Item> items;
    int32_t icount[kMaxPasses] = {0}, tcount[kMaxPasses] = {0};
    for (int l = 0; l < NL; ++l) {
      std::vector<std::pair<int32_t, int>> next_inter;
      for (int k = 0; k < D; ++k) {
        const int j = l * D + k;
        std::vector<Item> pass;
        for (size_t u = 0; u < su[l].size(); ++u) {
          const UnitProg &U = *su[l][u];
          for (int v = 0; v < U.n_pass[k]; ++v) {
            Item e{0xffff, 0xffff, 0, 0};
            if (k < D - 1 || l < NL - 1) {
              e.dst = (uint16_t)(base[l][k][u] + v);
              if (k == D - 1) next_inter.push_back({U.out_tile[v], base[l][k][u] + v});
            } else {
              e.dst = (uint16_t)(std::lower_bound(osorted.begin(), osorted.end(), U.out_tile[v]) - osorted.begin());
            }
            int got = 0;
            for (int b = 0; b < 2; ++b) {
              const int sidx = U.src[k][v][b];
              if (sidx < 0) continue;
              int slot;
              if (k > 0) {
                slot = base[l][k - 1][u] + sidx;
              } else if (l == 0) {
                slot = slot_of[base_in[u] + sidx];
              } else {
                // an intermediate tile of the previous level, by its global index
                const auto it = std::lower_bound(inter.begin(), inter.end(), std::make_pair(U.in_tile[sidx], -1));
                slot = it != inter.end() && it->first == U.in_tile[sidx] ? it->second : -1;
                if (slot < 0) {  // not produced in this chunk: cannot happen for whole units
                  if (fits) *fits = false;
                  slot = 0;
                }
              }
              if (got == 0) {
                e.src0 = (uint16_t)slot;
                e.ops = (uint16_t)U.op[k][v][b];
              } else {
                e.src1 = (uint16_t)slot;
                e.ops |= (uint16_t)(U.op[k][v][b] << 2);
              }
              ++got;
            }
            pass.push_back(e);
          }
        }
        // two-source items first, then by the delta and gamma of the first operator: a
        // step then rarely mixes one- and two-source fibres or operators of both deltas
        std::stable_sort(pass.begin(), pass.end(), [](const Item &x, const Item &y) {
          const int kx = ((x.src1 == 0xffff) << 2) | ((x.ops & 1) << 1) | ((x.ops >> 1) & 1);
          const int ky = ((y.src1 == 0xffff) << 2) | ((y.ops & 1) << 1) | ((y.ops >> 1) & 1);
          return kx < ky;
        });
        icount[j] = (int32_t)pass.size();
        for (const Item &e : pass) tcount[j] += e.src1 != 0xffff;
        items.insert(items.end(), pass.begin(), pass.end());
      }
      std::sort(next_inter.begin(), next_inter.end());
      inter.swap(next_inter);
    }
    std::vector<Run> oruns;
    for (size_t r = 0; r < osorted.size(); ++r) {
      if (r > 0 && osorted[r] == osorted[r - 1] + 1 && oruns.back().count < 0xffff)
        oruns.back().count++;
      else
        oruns.push_back(Run{osorted[r], (uint16_t)r, 1});
    }
    cd.blob_off = (int32_t)prog.blob.size();
    cd.n_pass = NP;
    int32_t header[kBlobHeader / 4] = {0};
    header[0] = NP;
    header[1] = cd.n_in;
    header[2] = (int32_t)oruns.size();
    for (int j = 0; j < NP; ++j) {
      header[4 + j] = icount[j];
      header[4 + kMaxPasses + j] = tcount[j];
    }
    const size_t ib = items.size() * sizeof(Item), ob = oruns.size() * sizeof(Run);
    const size_t bytes = (kBlobHeader + ib + ob + 15) & ~(size_t)15;
    prog.blob.resize(prog.blob.size() + bytes, 0);
    unsigned char *dstp = prog.blob.data() + cd.blob_off;
    std::memcpy(dstp, header, kBlobHeader);
    std::memcpy(dstp + kBlobHeader, items.data(), ib);
    std::memcpy(dstp + kBlobHeader + ib, oruns.data(), ob);
    cd.blob_bytes = (int32_t)bytes;
    prog.chunks.push_back(cd);
    cur.clear();
    tot = Tot();
  };
  auto push = [&](StepUnit &&m) {
    Tot t2 = tot;
    add(t2, m);
    if (!cur.empty() && !within(t2)) {
      flush();
      t2 = Tot();
      add(t2, m);
    }
    if (!within(t2) && fits) *fits = false;  // a unit alone exceeds the capacities
    cur.push_back(std::move(m));
    tot = t2;
  };

  // stages t, t-1, .. (trees st[0], st[1], ..): unit (A_top, B_bot) with A_top a box of
  // the A' level of stage t and B_bot one of the B level of stage t-NL+1.  Its level l
  // (stage t-l) units are (A, B) for the descendants A of A_top l levels down and B of
  // B_bot NL-1-l levels down; the tiles of the stages between levels stay in shared
  // memory.  The adjoint runs the levels in the reverse order.
  const int64_t n_top = (int64_t)st[0].csAp->size() - 1, n_bot = (int64_t)st[NL - 1].csB->size() - 1;
  std::vector<int32_t> As[kMaxLevels], Bs[kMaxLevels];
  for (int64_t iA = 0; iA < n_top; ++iA) {
    As[0].assign(1, (int32_t)iA);
    for (int l = 1; l < NL; ++l) {  // children along the A' levels of stages t, t-1, ..
      const std::vector<int32_t> &cs = *st[l - 1].csAp;
      As[l].clear();
      for (int32_t a : As[l - 1])
        for (int32_t c = cs[a]; c < cs[a + 1]; ++c) As[l].push_back(c);
    }
    for (int64_t iB = 0; iB < n_bot; ++iB) {
      Bs[NL - 1].assign(1, (int32_t)iB);
      for (int l = NL - 2; l >= 0; --l) {  // children along the B levels of stages t-NL+1, ..
        const std::vector<int32_t> &cs = *st[l + 1].csB;
        Bs[l].clear();
        for (int32_t b : Bs[l + 1])
          for (int32_t c = cs[b]; c < cs[b + 1]; ++c) Bs[l].push_back(c);
      }
      StepUnit m;
      for (int l = 0; l < NL; ++l) {
        std::vector<UnitProg> &dst = m.lev[adjoint ? NL - 1 - l : l];
        for (int32_t a : As[l])
          for (int32_t b : Bs[l]) dst.push_back(build_unit(D, st[l], a, b, adjoint));
      }
      push(std::move(m));
    }
  }
  flush();
  // the order in which the blocks of a launch take the chunks
  const size_t n = prog.chunks.size();
  std::vector<double> work(n);
  for (size_t c = 0; c < n; ++c) work[c] = chunk_work(prog.blob.data() + prog.chunks[c].blob_off, dim, p);
  const std::vector<size_t> order = schedule_chunks(work);
  std::vector<ChunkDesc> chunks(n);
  std::vector<int32_t> in_off(n);
  for (size_t c = 0; c < n; ++c) {
    chunks[c] = prog.chunks[order[c]];
    in_off[c] = prog.in_off[order[c]];
  }
  prog.chunks.swap(chunks);
  prog.in_off.swap(in_off);
  return prog;
}

std::vector<size_t> schedule_chunks(const std::vector<double> &work) {
  std::vector<size_t> order(work.size());
  std::iota(order.begin(), order.end(), (size_t)0);
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work[a] > work[b]; });
  return order;
}

double chunk_work(const unsigned char *blob_header, int dim, int p) {
  const int32_t *hdr = reinterpret_cast<const int32_t *>(blob_header);
  int64_t fib = 1;
  for (int d = 1; d < dim; ++d) fib *= p;
  double w = 1.0;
  for (int j = 0; j < hdr[0] && j < kMaxPasses; ++j) {
    const int64_t nf = hdr[4 + j] * fib, nf2 = hdr[4 + kMaxPasses + j] * fib;
    w += (double)((nf + 31) / 32 + (nf2 + 31) / 32) / kProgramWarps;
  }
  return w;
}

std::string validate_program(const StageProgram &prog, int dim, int p, ChunkCaps caps, int64_t in_tiles,
                             int64_t out_tiles) {
  (void)p;
  // every tile of the input stage is read by exactly one chunk and every tile of the
  // output stage written by exactly one (each pair of a stage belongs to one unit)
  std::vector<unsigned char> read((size_t)std::max<int64_t>(in_tiles, 0), 0), written((size_t)std::max<int64_t>(out_tiles, 0), 0);
  for (size_t ci = 0; ci < prog.chunks.size(); ++ci) {
    const ChunkDesc &c = prog.chunks[ci];
    if (c.blob_off < 0 || (c.blob_off & 15) || (size_t)c.blob_off + kBlobHeader > prog.blob.size())
      return "metadata blob out of range";
    const int32_t *hdr = reinterpret_cast<const int32_t *>(prog.blob.data() + c.blob_off);
    const int NP = hdr[0];
    if (NP != c.n_pass || NP < dim || NP > kMaxPasses || NP % dim != 0) return "metadata header mismatch";
    if (hdr[1] != c.n_in) return "metadata header mismatch";
    int need0 = c.n_in, need1 = 0;
    int64_t nitems = 0;
    for (int j = 0; j < NP; ++j) {
      const int ni = hdr[4 + j], n2 = hdr[4 + kMaxPasses + j];
      if (ni < 0 || n2 < 0 || n2 > ni) return "metadata header mismatch";
      if (j & 1) need0 = std::max(need0, ni);
      else need1 = std::max(need1, ni);
      nitems += ni;
    }
    const int nl = hdr[4 + NP - 1];
    if (c.n_in < 1 || need0 > caps.cap0 || need1 > caps.cap1 || nl > caps.max_out)
      return "chunk exceeds its shared-memory capacities";
    const int n_oruns = hdr[2];
    const int64_t need = (kBlobHeader + nitems * (int64_t)sizeof(Item) + n_oruns * (int64_t)sizeof(Run) + 15) & ~(int64_t)15;
    if (c.blob_bytes != need || c.blob_bytes > caps.meta_bytes || (size_t)c.blob_off + c.blob_bytes > prog.blob.size())
      return "metadata blob out of range";
    if (c.run_off < 0 || c.n_runs < 1 || (size_t)c.run_off + c.n_runs > prog.runs.size())
      return "run list out of range";
    int covered = 0;
    for (int r = 0; r < c.n_runs; ++r) {
      const Run &rn = prog.runs[c.run_off + r];
      if (rn.slot != covered || rn.count < 1 || rn.start < 0 || rn.start + (int64_t)rn.count > in_tiles)
        return "input run out of range";
      for (int q = 0; q < rn.count; ++q)
        if (read[rn.start + q]++) return "an input tile is read by two chunks";
      covered += rn.count;
    }
    if (covered != c.n_in) return "runs do not cover the inputs";
    const unsigned char *bp = prog.blob.data() + c.blob_off;
    const Item *items = reinterpret_cast<const Item *>(bp + kBlobHeader);
    const Run *oruns = reinterpret_cast<const Run *>(bp + kBlobHeader + nitems * sizeof(Item));
    covered = 0;
    for (int r = 0; r < n_oruns; ++r) {
      const Run &rn = oruns[r];
      if (rn.slot != covered || rn.count < 1 || rn.start < 0 || rn.start + (int64_t)rn.count > out_tiles)
        return "output run out of range";
      for (int q = 0; q < rn.count; ++q)
        if (written[rn.start + q]++) return "an output tile is written by two chunks";
      covered += rn.count;
    }
    if (covered != nl) return "output runs do not cover the outputs";
    int64_t off = 0;
    int nsrc = c.n_in;  // sources of pass j live in the previous pass's buffer
    for (int j = 0; j < NP; ++j) {
      const int ni = hdr[4 + j], n2 = hdr[4 + kMaxPasses + j];
      std::vector<char> seen(ni, 0);
      for (int i = 0; i < ni; ++i) {
        const Item &it = items[off + i];
        if (it.src0 >= nsrc) return "item source 0 out of range";
        if ((i < n2) != (it.src1 != 0xffff)) return "two-source items do not lead the pass";
        if (it.src1 != 0xffff && it.src1 >= nsrc) return "item source 1 out of range";
        if (it.ops >= (it.src1 != 0xffff ? 16 : 4)) return "operator out of range";
        if (it.dst >= ni || seen[it.dst]) return "item destination out of range or repeated";
        seen[it.dst] = 1;
      }
      off += ni;
      nsrc = ni;
    }
  }
  for (unsigned char v : read)
    if (!v) return "an input tile is read by no chunk";
  for (unsigned char v : written)
    if (!v) return "an output tile is written by no chunk";
  return "";
}

}  // namespace bfly
