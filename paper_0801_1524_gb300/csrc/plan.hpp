// Host side of the plan: trees, per-level box lists, operator tables, work chunks.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace bfly {

// One block of work of the recursive step: a run of consecutive units, compiled on the
// host into per-pass item lists (see make_step_program).  A step applies one level of the
// recursion (D passes, one per axis) or two consecutive levels (2D passes; the tiles of the
// level between them stay in shared memory).  Its metadata blob (a 64-byte header
// {n_pass, n_in, n_out_runs, 0, n_item[kMaxPasses], n_two[kMaxPasses]} (n_two: the leading
// two-source items of each pass), the items of every pass, then the output runs, padded
// to 16 bytes) is copied to shared memory in one piece; its inputs are copied run by run,
// its outputs written back run by run.
constexpr int kBlobHeader = 64;
constexpr int kMaxPasses = 6;
constexpr int kMaxLevels = 3;  // stages per launch (2D; 3D: one)
// Consumer warps of a recursive-step block, which split every pass of a chunk.
constexpr int kProgramWarps = 7;
struct ChunkDesc {
  int32_t blob_off;   // byte offset of the blob in StageProgram::blob (16-byte aligned)
  int32_t blob_bytes; // multiple of 16
  int32_t run_off;    // first run in StageProgram::runs
  int32_t n_runs;
  int32_t n_in;       // input tiles (the runs' total)
  int32_t n_pass;     // passes (the last writes the outputs)
  int32_t pad[2];
};
static_assert(sizeof(ChunkDesc) == 32, "ChunkDesc is uploaded as 32 bytes");

// One output tile of a pass: the sum over one or two source tiles of the previous pass
// (pass 0: input tiles) of C^{op} applied along the pass's axis, stored to slot dst.  A
// pass lists its two-source items first; every lane of a step takes one fibre of the
// flat list of the pass's fibres, with its own item's operators.
struct Item {
  uint16_t src0, src1;  // chunk-local source slots; src1 = 0xffff when absent
  uint16_t dst;         // destination slot (last pass: staging slot of the output run)
  uint16_t ops;         // op of src0 in bits 0-1, op of src1 in bits 2-3 (op = gamma*2 + delta)
};
static_assert(sizeof(Item) == 8, "Item is uploaded as 8 bytes");

// A run of consecutive tiles: global tiles [start, start + count) <-> chunk-local slots
// [slot, slot + count) (inputs: copied in; outputs: written back from the staging slots).
struct Run {
  int32_t start;
  uint16_t slot, count;
};
static_assert(sizeof(Run) == 8, "Run is uploaded as 8 bytes");

// A chunk of a batched launch: the chunk and the buffers of the plan it belongs to.
struct BatchEntry {
  ChunkDesc d;
  const unsigned char *blob;
  const Run *runs;
  const void *in;
  void *out;
  int64_t in_rhs, out_rhs;  // elements between right-hand sides of the plan's buffers
};
static_assert(sizeof(BatchEntry) == 80, "BatchEntry is uploaded as 80 bytes");

struct StageProgram {
  std::vector<ChunkDesc> chunks;
  std::vector<unsigned char> blob;  // per chunk: header, Item[], Run[n_out_runs]
  std::vector<Run> runs;
  // host-side copies used for validation and statistics
  std::vector<int32_t> in_tiles;    // global tile of every input slot, chunk after chunk
  std::vector<int32_t> in_off;      // per chunk: first entry of in_tiles
};

// Shared-memory capacities of one block, in tiles: pass j reads the buffer pass j-1 wrote
// and writes the scratch buffer (even j) or the input buffer (odd j); the input buffer
// first holds the inputs.  At most max_out outputs; a metadata blob of at most meta_bytes.
struct ChunkCaps {
  int cap0, cap1, max_out, meta_bytes;
};

// A quadtree (octree) over [0,2^L]^dim with unit leaves, non-empty boxes only, boxes of
// every level in Morton order so that the children of a box are consecutive.  The points
// are those of the caller scaled by s = sqrt(2^L / N) (s = 1 when N = 2^L), so that
// x.k/N = x'.k'/2^L: the transform of any N is the one of 2^L on the scaled points.
struct HostTree {
  int dim = 0, L = 0;
  int64_t n = 0;
  std::vector<int32_t> perm;              // sorted position -> caller index
  std::vector<double> off;                // [n][dim] scaled offset from the leaf corner, [0,1]
  std::vector<int32_t> point_leaf;        // sorted position -> leaf number
  std::vector<int32_t> leaf_start;        // [nleaf+1] point range of every leaf
  std::vector<std::vector<int32_t>> idx;  // idx[s]: [n_s][dim] box index per axis
  std::vector<std::vector<int32_t>> cs;   // cs[s]: [n_s+1] child range in level s+1
  int64_t nbox(int s) const { return (int64_t)idx[s].size() / dim; }
  int nchild(int s, int64_t i) const { return cs[s][i + 1] - cs[s][i]; }
};

// Sec. 2.2 step 1.  pts: [n][dim] in [0, N]; a coordinate v lies in leaf floor(v s)
// (clamped to 2^L - 1).  Returns an error message or "".
std::string build_tree(HostTree &T, int dim, int L, double N, double scale, int64_t n, const double *pts);

// Transfer operators of the recursive step (eqs. M1 and E1 combined) for the rescaled
// charges g^{AB}_m = e^{2 pi i a m/q} f^{AB}_m (a the index of A along the axis), per
// axis:  C^{(gamma,delta)}[m][l] = w_m(tau_l) e^{2 pi i gamma tau_l},
// tau_l = (delta + l/q)/2, gamma the bit of A within A', delta that of Bc within B.
// The factors of the transfer operators, C^{(gamma,delta)} = W(delta) diag(phi_gamma)
// (phi_0 = 1), as interleaved (re, im) doubles: W [2][p][p] (delta, row, column) and
// phi [2][p] = phi_1 for delta = 0, 1.  adjoint = true gives the factors of the
// conjugate-transposed operators, diag(conj phi_gamma) W(delta)^H: W^H and conj(phi_1).
void transfer_factors(int p, bool adjoint, double *W /* 2*p*p*2 */, double *phi /* 2*p*2 */);

// Lagrange weights of the leaf step, w_m(tau) = (G^{-1} v(tau))_m, m = 0..p-1, for
// G_{ll'} = e^{2 pi i l l'/q^2}, v(tau)_l = e^{2 pi i l tau/q}, tau in leaf widths.
void leaf_weights(int p, double tau, double *w /* 2p doubles */);

// The trees of stage t of the recursive step:
//   csAp : children of the A' boxes (T_X level L-t-1 -> L-t), xidx: box indices of level L-t
//   csB  : children of the B boxes (T_K level t -> t+1),       kidx: box indices of level t+1
struct StageTrees {
  const std::vector<int32_t> *csAp, *xidx, *csB, *kidx;
};

// The recursive step as chunk programs, for the `levels` consecutive stages t, t-1, ..
// (st[l]: the trees of stage t-l; levels * dim <= kMaxPasses) in one launch.  Forward, a
// unit (A', B) of stage t reads the tiles f^{A'Bc} of the children Bc of B and writes
// f^{AB} for the children A of A'; adjoint: reads f^{AB} of the children A, writes
// f^{A'Bc}.  The operator of every (A, Bc) pair is (x)_d C^{(gamma_d(A), delta_d(Bc))};
// passes apply one axis each and sum, before each axis, the sources that agree on all
// bits still to be applied (sum factorisation).  Several levels: unit (A_top, B_bot)
// (A_top on the A' level of stage t, B_bot on the B level of the last stage) groups, for
// every level l, the stage-(t-l) units (A, B) with A a descendant of A_top l levels down
// and B one of B_bot levels-1-l levels down (the adjoint runs the levels in reverse);
// the tiles of the stages between levels are not written out.
// The chunks are runs of consecutive units within the capacities, listed in the order of
// schedule_chunks.  *fits (optional) becomes false when a single unit exceeds them.
StageProgram make_step_program(int dim, int p, const StageTrees *st, int levels, bool adjoint, ChunkCaps caps,
                               bool *fits = nullptr);

// The order in which the persistent blocks of a launch take the chunks (indices into
// work): decreasing work, so that the blocks that finish first take the smallest chunks
// last (longest processing time first).
std::vector<size_t> schedule_chunks(const std::vector<double> &work);

// Estimated work of a chunk from its blob header: one unit per chunk (waits, barriers)
// plus, per pass, the 32-lane steps of its fibres (two-source fibres count twice) over
// the kProgramWarps consumer warps that share them.
double chunk_work(const unsigned char *blob_header, int dim, int p);

// Checks every index of a compiled step program against the capacities it was compiled
// for and the number of tiles of its input and output stage buffers, and that every input
// tile is read and every output tile written by exactly one chunk; returns "" or a
// description of the first violation.
std::string validate_program(const StageProgram &prog, int dim, int p, ChunkCaps caps, int64_t in_tiles,
                             int64_t out_tiles);

}  // namespace bfly
