// Host side of the plan: trees, per-level box lists, operator tables, work chunks.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace bfly {

// Capacity of one block of work of the recursive step (one chunk).
constexpr int kMaxUnits = 256;   // (A', B) units per chunk
constexpr int kMaxIn = 256;      // input charge tiles per chunk
constexpr int kMaxOut = 256;     // output charge tiles per chunk

// A chunk: `nu` consecutive units starting at unit u0 = iAp * nB + iB.  When nu == 1 the
// chunk may cover only outputs [o_lo, o_hi) of that unit (a unit too big for one block).
struct Chunk {
  int64_t u0;
  int32_t nu;
  int16_t o_lo, o_hi;
};
static_assert(sizeof(Chunk) == 16, "Chunk is uploaded as 16 bytes");

// A quadtree (octree) over [0,N]^dim with unit leaves, non-empty boxes only, boxes of
// every level in Morton order so that the children of a box are consecutive.
struct HostTree {
  int dim = 0, L = 0;
  int64_t n = 0;
  std::vector<int32_t> perm;              // sorted position -> caller index
  std::vector<double> off;                // [n][dim] offset from the leaf corner, [0,1]
  std::vector<int32_t> point_leaf;        // sorted position -> leaf number
  std::vector<int32_t> leaf_start;        // [nleaf+1] point range of every leaf
  std::vector<std::vector<int32_t>> idx;  // idx[s]: [n_s][dim] box index per axis
  std::vector<std::vector<int32_t>> cs;   // cs[s]: [n_s+1] child range in level s+1
  int64_t nbox(int s) const { return (int64_t)idx[s].size() / dim; }
  int nchild(int s, int64_t i) const { return cs[s][i + 1] - cs[s][i]; }
};

// Sec. 2.2 step 1.  pts: [n][dim] in [0, 2^L]; returns an error message or "".
std::string build_tree(HostTree &T, int dim, int L, int64_t n, const double *pts);

// Transfer operators of the recursive step (eqs. M1 and E1 combined), per axis:
//   T^{(alpha,delta)}[m][l] , alpha = a mod 2(p-1), delta = child offset bit,
// stored [4(p-1)][p][p] as interleaved (re, im) doubles, op index alpha*2 + delta.
// adjoint = true stores the conjugate transpose of every operator.
std::vector<double> transfer_table(int p, bool adjoint);

// Lagrange weights of the leaf step, w_m(tau) = (G^{-1} v(tau))_m, m = 0..p-1.
void leaf_weights(int p, double tau, double *w /* 2p doubles */);

// Chunks of the recursive step at one stage.  The unit (A', B) has nout outputs and nin
// inputs: forward nin = children of B, nout = children of A'; adjoint the reverse.  Every
// chunk needs (inputs + outputs*inputs) tiles of shared memory.
std::vector<Chunk> make_chunks(const std::vector<int32_t> &csAp, const std::vector<int32_t> &csB,
                               bool adjoint, int tile_cap);

}  // namespace bfly
