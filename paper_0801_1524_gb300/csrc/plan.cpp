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

}  // namespace

StageProgram make_stage_program(int dim, int p, const std::vector<int32_t> &csAp,
                                const std::vector<int32_t> &xidx, const std::vector<int32_t> &csB,
                                const std::vector<int32_t> &kidx, bool adjoint, ChunkCaps caps) {
  StageProgram prog;
  const int q = p - 1;
  const int D = dim;
  const int64_t nAp = (int64_t)csAp.size() - 1, nB = (int64_t)csB.size() - 1;
  const int64_t nBc = (int64_t)kidx.size() / dim;
  const int64_t in_row = adjoint ? nB : nBc, out_row = adjoint ? nBc : nB;
  auto lo = [](int k) { return (1 << (k + 1)) - 1; };     // bits 0..k
  auto hi = [&](int k) { return ((1 << D) - 1) & ~lo(k); };  // bits k+1..D-1

  int tot_in = 0, tot[3] = {0, 0, 0};
  std::vector<UnitProg> units;
  auto flush = [&]() {
    if (units.empty()) return;
    ChunkDesc cur{};
    cur.n_in = tot_in;
    for (int k = 0; k < 3; ++k) cur.n_item[k] = k < D ? tot[k] : 0;
    // inputs of the chunk in global order: slot = rank, so that runs are contiguous
    std::vector<std::pair<int32_t, int>> order;  // (global tile, unit-local key index)
    std::vector<int> base_in(units.size());
    int bi = 0;
    for (size_t u = 0; u < units.size(); ++u) {
      base_in[u] = bi;
      for (int i = 0; i < units[u].n_in; ++i) order.push_back({units[u].in_tile[i], bi + i});
      bi += units[u].n_in;
    }
    std::vector<std::pair<int32_t, int>> sorted = order;
    std::sort(sorted.begin(), sorted.end());
    std::vector<int> slot_of(order.size());
    for (size_t r = 0; r < sorted.size(); ++r) slot_of[sorted[r].second] = (int)r;
    prog.in_off.push_back((int32_t)prog.in_tiles.size());
    cur.run_off = (int32_t)prog.runs.size();
    for (size_t r = 0; r < sorted.size(); ++r) {
      prog.in_tiles.push_back(sorted[r].first);
      if (r > 0 && sorted[r].first == sorted[r - 1].first + 1 && prog.runs.back().count < 0xffff)
        prog.runs.back().count++;
      else
        prog.runs.push_back(Run{sorted[r].first, (uint16_t)r, 1});
    }
    cur.n_runs = (int32_t)prog.runs.size() - cur.run_off;
    // pass tiles numbered unit by unit
    std::vector<int> base[3];
    for (int k = 0; k < 3; ++k) base[k].resize(units.size());
    int bk[3] = {0, 0, 0};
    for (size_t u = 0; u < units.size(); ++u)
      for (int k = 0; k < D; ++k) {
        base[k][u] = bk[k];
        bk[k] += units[u].n_pass[k];
      }
    // items pass by pass; the last pass's destination is the staging slot of its output,
    // numbered in global order so that outputs form contiguous runs
    std::vector<int32_t> outs;
    for (size_t u = 0; u < units.size(); ++u)
      for (int v = 0; v < units[u].n_pass[D - 1]; ++v) outs.push_back(units[u].out_tile[v]);
    std::vector<int32_t> osorted = outs;
    std::sort(osorted.begin(), osorted.end());
    std::vector<Task> tasks;
    std::vector<Group> groups;
    int32_t counts[6] = {0, 0, 0, 0, 0, 0}, gcounts[6] = {0, 0, 0, 0, 0, 0};
    int fib = 1;  // fibres of one tile along one axis
    for (int d = 0; d + 1 < D; ++d) fib *= p;
    int oi = 0;
    for (int k = 0; k < D; ++k) {
      std::vector<Task> ph[2];
      for (size_t u = 0; u < units.size(); ++u) {
        const UnitProg &U = units[u];
        for (int v = 0; v < U.n_pass[k]; ++v) {
          uint16_t dst;
          if (k == D - 1) {
            const int32_t g = outs[oi++];
            dst = (uint16_t)(std::lower_bound(osorted.begin(), osorted.end(), g) - osorted.begin());
          } else {
            dst = (uint16_t)(base[k][u] + v);
          }
          int got = 0;
          for (int j = 0; j < 2; ++j) {
            const int sidx = U.src[k][v][j];
            if (sidx < 0) continue;
            const int slot = k == 0 ? slot_of[base_in[u] + sidx] : base[k - 1][u] + sidx;
            ph[got].push_back(Task{(uint16_t)slot, dst, (uint16_t)U.op[k][v][j], 0});
            ++got;
          }
        }
      }
      for (int f = 0; f < 2; ++f) {
        std::stable_sort(ph[f].begin(), ph[f].end(), [](const Task &x, const Task &y) { return x.op < y.op; });
        counts[2 * k + f] = (int32_t)ph[f].size();
        int steps = 0;
        for (size_t i = 0; i < ph[f].size();) {
          size_t j = i;
          while (j < ph[f].size() && ph[f][j].op == ph[f][i].op) ++j;
          const int n = (int)(j - i);
          groups.push_back(Group{(uint16_t)i, (uint16_t)n, ph[f][i].op, (uint16_t)steps});
          steps += (n * fib + 31) / 32;
          ++gcounts[2 * k + f];
          i = j;
        }
        tasks.insert(tasks.end(), ph[f].begin(), ph[f].end());
      }
    }
    std::vector<Run> oruns;
    for (size_t r = 0; r < osorted.size(); ++r) {
      if (r > 0 && osorted[r] == osorted[r - 1] + 1 && oruns.back().count < 0xffff)
        oruns.back().count++;
      else
        oruns.push_back(Run{osorted[r], (uint16_t)r, 1});
    }
    cur.blob_off = (int32_t)prog.blob.size();
    int32_t header[16] = {0};
    for (int i = 0; i < 6; ++i) {
      header[i] = counts[i];
      header[6 + i] = gcounts[i];
    }
    header[12] = cur.n_in;
    header[13] = (int32_t)oruns.size();
    const size_t ib = tasks.size() * sizeof(Task), gb = groups.size() * sizeof(Group);
    const size_t ob = oruns.size() * sizeof(Run);
    const size_t bytes = (64 + ib + gb + ob + 15) & ~(size_t)15;
    prog.blob.resize(prog.blob.size() + bytes, 0);
    unsigned char *dstp = prog.blob.data() + cur.blob_off;
    std::memcpy(dstp, header, 64);
    std::memcpy(dstp + 64, tasks.data(), ib);
    std::memcpy(dstp + 64 + ib, groups.data(), gb);
    std::memcpy(dstp + 64 + ib + gb, oruns.data(), ob);
    cur.blob_bytes = (int32_t)bytes;
    prog.chunks.push_back(cur);
    units.clear();
    tot_in = 0;
    tot[0] = tot[1] = tot[2] = 0;
  };

  for (int64_t iAp = 0; iAp < nAp; ++iAp) {
    const int a0 = csAp[iAp], a1 = csAp[iAp + 1];
    int apar[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) apar[d] = xidx[(int64_t)a0 * D + d] >> 1;
    auto alpha = [&](int d, int bit) { return (2 * apar[d] + bit) % (2 * q); };
    for (int64_t iB = 0; iB < nB; ++iB) {
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
        U.in_tile[i] = adjoint ? (int32_t)((int64_t)gtile[i] * in_row + iB)
                               : (int32_t)(iAp * in_row + dtile[i]);
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
            const int S = (K & ~(1 << k)) | (b << k);
            int found = -1;
            if (k == 0) {
              for (int i = 0; i < n_in; ++i)
                if (U.in_key[i] == S) found = i;  // input keys are all in-side bits
            } else {
              for (int j = 0; j < U.n_pass[k - 1]; ++j)
                if (U.key[k - 1][j] == S) found = j;
            }
            U.src[k][v][b] = found;
            // forward: alpha from the output (gamma) bit, delta = b; adjoint: alpha from
            // the input (gamma) bit b, delta = the output bit
            U.op[k][v][b] = adjoint ? alpha(k, b) * 2 + obit : alpha(k, obit) * 2 + b;
          }
        }
      }
      for (int v = 0; v < U.n_pass[D - 1]; ++v) {
        // the last pass's keys are output keys: find that output's tile
        for (int o = 0; o < n_out; ++o)
          if (okey[o] == U.key[D - 1][v])
            U.out_tile[v] = adjoint ? (int32_t)(iAp * out_row + dtile[o])
                                    : (int32_t)((int64_t)gtile[o] * out_row + iB);
      }
      // capacity: buffer 0 holds inputs (and pass 1 in 3D), buffer 1 pass 0
      const int need0 = std::max(tot_in + U.n_in, D == 3 ? tot[1] + U.n_pass[1] : 0);
      const int need1 = tot[0] + U.n_pass[0];
      const int needo = tot[D - 1] + U.n_pass[D - 1];
      // header, two tasks and up to two groups per item, one run per output
      const int needb = 64 + 32 * (need1 + (D == 3 ? tot[1] + U.n_pass[1] : 0) + needo) + 8 * needo + 15;
      if (!units.empty() && (need0 > caps.cap0 || need1 > caps.cap1 || needo > caps.max_out ||
                             needb > caps.meta_bytes))
        flush();
      units.push_back(U);
      tot_in += U.n_in;
      for (int k = 0; k < D; ++k) tot[k] += U.n_pass[k];
    }
  }
  flush();
  return prog;
}

std::string validate_program(const StageProgram &prog, int dim, ChunkCaps caps, int64_t in_tiles,
                             int64_t out_tiles) {
  for (size_t ci = 0; ci < prog.chunks.size(); ++ci) {
    const ChunkDesc &c = prog.chunks[ci];
    const int n0 = c.n_item[0], n1 = dim == 3 ? c.n_item[1] : 0, nl = c.n_item[dim - 1];
    const int stage_cap = dim == 3 ? caps.cap1 : caps.cap0;  // outputs are staged there
    if (c.n_in < 1 || c.n_in > caps.cap0 || n0 > caps.cap1 || n1 > caps.cap0 || nl > caps.max_out ||
        nl > stage_cap)
      return "chunk exceeds its shared-memory capacities";
    if (c.blob_off < 0 || (c.blob_off & 15) || (size_t)c.blob_off + 64 > prog.blob.size())
      return "metadata blob out of range";
    const int32_t *hdr = reinterpret_cast<const int32_t *>(prog.blob.data() + c.blob_off);
    int64_t ntasks = 0, ngroups = 0;
    for (int k = 0; k < dim; ++k) {
      if (hdr[2 * k] != c.n_item[k] || hdr[2 * k + 1] < 0 || hdr[2 * k + 1] > hdr[2 * k])
        return "metadata header mismatch";
      ntasks += hdr[2 * k] + hdr[2 * k + 1];
      ngroups += hdr[6 + 2 * k] + hdr[6 + 2 * k + 1];
    }
    if (hdr[12] != c.n_in) return "metadata header mismatch";
    const int n_oruns = hdr[13];
    const int64_t need = (64 + ntasks * (int64_t)sizeof(Task) + ngroups * (int64_t)sizeof(Group) +
                          n_oruns * (int64_t)sizeof(Run) + 15) & ~(int64_t)15;
    if (c.blob_bytes != need || c.blob_bytes > caps.meta_bytes || (size_t)c.blob_off + c.blob_bytes > prog.blob.size())
      return "metadata blob out of range";
    if (c.run_off < 0 || c.n_runs < 1 || (size_t)c.run_off + c.n_runs > prog.runs.size())
      return "run list out of range";
    int covered = 0;
    for (int r = 0; r < c.n_runs; ++r) {
      const Run &rn = prog.runs[c.run_off + r];
      if (rn.slot != covered || rn.count < 1 || rn.start < 0 || rn.start + (int64_t)rn.count > in_tiles)
        return "input run out of range";
      covered += rn.count;
    }
    if (covered != c.n_in) return "runs do not cover the inputs";
    const Task *tasks = reinterpret_cast<const Task *>(prog.blob.data() + c.blob_off + 64);
    const Group *groups = reinterpret_cast<const Group *>(tasks + ntasks);
    const Run *oruns = reinterpret_cast<const Run *>(groups + ngroups);
    covered = 0;
    for (int r = 0; r < n_oruns; ++r) {
      const Run &rn = oruns[r];
      if (rn.slot != covered || rn.count < 1 || rn.start < 0 || rn.start + (int64_t)rn.count > out_tiles)
        return "output run out of range";
      covered += rn.count;
    }
    if (covered != nl) return "output runs do not cover the outputs";
    int off = 0, goff = 0;
    int nsrc = c.n_in;  // sources of pass k live in the previous pass's buffer
    for (int k = 0; k < dim; ++k) {
      for (int f = 0; f < 2; ++f) {
        const int nt = hdr[2 * k + f], ng = hdr[6 + 2 * k + f];
        std::vector<char> seen(c.n_item[k], 0);
        for (int i = 0; i < nt; ++i) {
          const Task &tk = tasks[off + i];
          if (tk.src >= nsrc) return "task source out of range";
          if (tk.dst >= c.n_item[k] || seen[tk.dst]) return "task destination out of range or repeated";
          if (tk.op >= 64) return "task operator out of range";
          seen[tk.dst] = 1;
        }
        int covered_t = 0;
        for (int g = 0; g < ng; ++g) {
          const Group &gr = groups[goff + g];
          if (gr.task_begin != covered_t || gr.n_tasks < 1 || gr.task_begin + gr.n_tasks > nt)
            return "operator groups do not tile the tasks";
          for (int i = 0; i < gr.n_tasks; ++i)
            if (tasks[off + gr.task_begin + i].op != gr.op) return "task outside its operator group";
          covered_t += gr.n_tasks;
        }
        if (covered_t != nt) return "operator groups do not cover the tasks";
        off += nt;
        goff += ng;
      }
      nsrc = c.n_item[k];
    }
  }
  return "";
}

}  // namespace bfly
