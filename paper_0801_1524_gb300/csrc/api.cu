// C ABI of the butterfly (include/bfly.h): plan creation, upload and the execution entry
// points.  Every step of the transform runs in the kernels of this library.
#include <algorithm>
#include <atomic>
#include <deque>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/bfly.h"
#include "kernels.hpp"
#include "plan.hpp"

using bfly::ChunkCaps;
using bfly::StageProgram;
using bfly::HostTree;
using bfly::KernelSet;

namespace {

thread_local std::string g_err;

bfly_status fail(bfly_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

#define BFLY_CUDA(call)                                                                    \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? BFLY_ERR_OUT_OF_MEMORY : BFLY_ERR_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

const KernelSet *select_kernels(int p, int prec, int dim) {
  switch (p) {
    case 3: return bfly::kernels_p3(prec, dim);
    case 5: return bfly::kernels_p5(prec, dim);
    case 7: return bfly::kernels_p7(prec, dim);
    case 9: return bfly::kernels_p9(prec, dim);
    default: return nullptr;
  }
}

}  // namespace

#include "plan_state.hpp"

using bfly_state::flow_args;
using bfly_state::level_args;
using bfly_state::point_args;

namespace {

// Collects the plan's device arrays, then makes one allocation and uploads them.
struct Arena {
  struct Item {
    void **slot;
    size_t bytes;
    const void *host;
  };
  std::vector<Item> items;
  size_t total = 0;
  void add(void **slot, size_t bytes, const void *host = nullptr) {
    items.push_back({slot, bytes, host});
    total += (bytes + 255) & ~(size_t)255;
  }
  template <typename T>
  void add_vec(T **slot, const std::vector<T> &v) {
    add(reinterpret_cast<void **>(slot), v.size() * sizeof(T), v.data());
  }
};

// Levels below the root: the smallest L with 2^L >= N (up to a relative 1e-12), 0 for
// N <= 1.  The points are scaled by sqrt(2^L / N) so that the transform is the one of
// N' = 2^L (x.k/N = x'.k'/N').
int levels_for(double N) {
  if (!(N > 1.0)) return 0;
  return (int)std::ceil(std::log2(N) - 1e-12);
}

// Output runs of chunk c of a compiled step program (read from its metadata blob).
std::pair<const bfly::Run *, int> output_runs(const bfly::StageProgram &pg, size_t c) {
  const unsigned char *bp = pg.blob.data() + pg.chunks[c].blob_off;
  const int32_t *hdr = reinterpret_cast<const int32_t *>(bp);
  int64_t n_items = 0;
  for (int j = 0; j < hdr[0]; ++j) n_items += hdr[4 + j];
  return {reinterpret_cast<const bfly::Run *>(bp + bfly::kBlobHeader + n_items * sizeof(bfly::Item)), hdr[2]};
}

// The single-launch sweep of one direction (flow step k: plan step k forward, S-1-k for
// the adjoint).  Its entries are all chunks of all steps, step after step; a chunk of step
// k reads tiles that chunks of step k-1 write (its sources), which come before it, as the
// kernel's progress requires.  Returns an error message or "".
std::string build_flow(bfly_plan_t P, bool adjoint, int blocks, bfly_plan_s::Flow &F) {
  const int S = (int)P->steps.size();
  F = bfly_plan_s::Flow{};
  std::vector<const bfly::StageProgram *> pg(S);
  std::vector<int64_t> in_tiles(S);
  std::vector<int32_t> base(S + 1, 0);
  for (int k = 0; k < S; ++k) {
    const int s = adjoint ? S - 1 - k : k;
    const bfly_plan_s::Step &st = P->steps[s];
    pg[k] = adjoint ? &P->progA[s] : &P->progF[s];
    in_tiles[k] = adjoint ? P->pairs[st.t - st.levels + 1] : P->pairs[st.t + 1];
    base[k + 1] = base[k] + (int32_t)pg[k]->chunks.size();
  }
  const int32_t N = base[S];
  std::vector<int32_t> src_off((size_t)N + 1, 0), src;  // sources of every node (node ids)
  std::vector<int32_t> owner, d;
  for (int k = 0; k < S; ++k) {
    if (k > 0) {
      owner.assign((size_t)in_tiles[k], -1);
      for (size_t c = 0; c < pg[k - 1]->chunks.size(); ++c) {
        const auto runs = output_runs(*pg[k - 1], c);
        for (int j = 0; j < runs.second; ++j) {
          const bfly::Run r = runs.first[j];
          if (r.start < 0 || (int64_t)r.start + r.count > in_tiles[k]) return "output run outside its stage";
          for (int q = 0; q < r.count; ++q) owner[(size_t)r.start + q] = base[k - 1] + (int32_t)c;
        }
      }
    }
    for (size_t c = 0; c < pg[k]->chunks.size(); ++c) {
      const bfly::ChunkDesc &cd = pg[k]->chunks[c];
      const int32_t n = base[k] + (int32_t)c;
      d.clear();
      for (int j = 0; k > 0 && j < cd.n_runs; ++j) {
        const bfly::Run r = pg[k]->runs[(size_t)cd.run_off + j];
        if (r.start < 0 || (int64_t)r.start + r.count > in_tiles[k]) return "input run outside its stage";
        for (int q = 0; q < r.count; ++q) {
          const int32_t o = owner[(size_t)r.start + q];
          if (o < 0) return "an input tile that no chunk of the step before writes";
          if (d.empty() || d.back() != o) d.push_back(o);
        }
      }
      std::sort(d.begin(), d.end());
      d.erase(std::unique(d.begin(), d.end()), d.end());
      src.insert(src.end(), d.begin(), d.end());
      src_off[(size_t)n + 1] = (int32_t)src.size();
    }
  }
  // the order: step after step; within a step by the last of the chunk's sources in the
  // launch's order, in groups of half the grid's blocks (the chunks whose sources were
  // taken early come first, for the blocks that reach the step while the step before it
  // drains), the step's own order (decreasing work) within a group (groups of a quarter,
  // a whole or two grids, or none, measured slower on curve8192)
  std::vector<int32_t> order;
  order.reserve((size_t)N);
  std::vector<int32_t> pos((size_t)N, -1);
  for (int k = 0; k < S; ++k) {
    const int32_t n0 = base[k], n1 = base[k + 1];
    std::vector<int32_t> step_nodes;
    for (int32_t n = n0; n < n1; ++n) step_nodes.push_back(n);
    std::vector<int64_t> key((size_t)(n1 - n0), 0);
    for (int32_t n = n0; n < n1; ++n) {
      int32_t last = -1;
      for (int32_t j = src_off[n]; j < src_off[n + 1]; ++j) last = std::max(last, pos[src[j]]);
      key[n - n0] = last < 0 ? 0 : last / std::max(blocks / 2, 1);
    }
    std::stable_sort(step_nodes.begin(), step_nodes.end(),
                     [&](int32_t x, int32_t y) { return key[x - n0] < key[y - n0]; });
    for (int32_t n : step_nodes) {
      pos[n] = (int32_t)order.size();
      order.push_back(n);
    }
  }
  // entries in that order
  F.dep_off.assign(1, 0);
  F.first_use.assign((size_t)N, -1);
  F.nodes.reserve((size_t)N);
  for (int32_t i = 0; i < N; ++i) {
    const int32_t n = order[i];
    const int k = (int)(std::upper_bound(base.begin(), base.end(), n) - base.begin()) - 1;
    F.nodes.push_back({k, n - base[k]});
    d.clear();
    for (int32_t j = src_off[n]; j < src_off[n + 1]; ++j) d.push_back(pos[src[j]]);
    std::sort(d.begin(), d.end());
    for (int32_t x : d) {
      if (x >= i) return "a chunk ordered before one of its sources";
      if (F.first_use[x] < 0) F.first_use[x] = i;
    }
    F.dep_idx.insert(F.dep_idx.end(), d.begin(), d.end());
    F.dep_off.push_back((int32_t)F.dep_idx.size());
  }
  F.n_entries = N;
  // rows {count, the first kFlowDepRow - 1 sources, -1 ...}
  const int K = bfly::kFlowDepRow;
  F.deps.assign((size_t)N * K, -1);
  for (int32_t e = 0; e < N; ++e) {
    const int32_t n = F.dep_off[e + 1] - F.dep_off[e];
    F.deps[(size_t)e * K] = n;
    std::copy(F.dep_idx.begin() + F.dep_off[e], F.dep_idx.begin() + F.dep_off[e] + std::min(n, K - 1),
              F.deps.begin() + (size_t)e * K + 1);
  }
  return "";
}

std::string build_flows(bfly_plan_t P) {
  const int blocks = P->level_grid > 0 ? P->level_grid : 456;
  std::string bad = build_flow(P, false, blocks, P->flowF);
  if (bad.empty()) bad = build_flow(P, true, blocks, P->flowA);
  return bad;
}

// Uploads the launch entries of both directions (they hold device pointers of the plan's
// allocation) and clears the flags, epochs and work counters of the single-launch sweep.
cudaError_t upload_flows(bfly_plan_t P) {
  const int S = (int)P->steps.size();
  P->fbuf[0] = P->buf[0];
  P->fbuf[S] = P->buf[1];
  for (int dir = 0; dir < 2; ++dir) {
    bfly_plan_s::Flow &F = dir ? P->flowA : P->flowF;
    std::vector<bfly::BatchEntry> ent;
    ent.reserve((size_t)F.n_entries);
    for (const auto &node : F.nodes) {
      const int s = dir ? S - 1 - node.first : node.first;
      const bfly_plan_s::Step &st = P->steps[s];
      const int64_t hi = P->pairs[st.t + 1] * P->TS, lo = P->pairs[st.t - st.levels + 1] * P->TS;
      const bfly::StageProgram &pg = dir ? P->progA[s] : P->progF[s];
      const bfly_plan_s::DevProg &dp = dir ? P->dA[s] : P->dF[s];
      bfly::BatchEntry be{};
      be.d = pg.chunks[(size_t)node.second];
      be.blob = dp.blob;
      be.runs = dp.runs;
      be.in = dir ? P->fbuf[s + 1] : P->fbuf[s];
      be.out = dir ? P->fbuf[s] : P->fbuf[s + 1];
      be.in_rhs = dir ? lo : hi;
      be.out_rhs = dir ? hi : lo;
      ent.push_back(be);
    }
    if ((int)ent.size() != F.n_entries) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpy(F.entries, ent.data(), ent.size() * sizeof(bfly::BatchEntry), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(F.flags, 0, (size_t)F.n_entries * P->max_nrhs * sizeof(unsigned));
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemset(P->epoch, 0, 2 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(P->flow_sched, 0, 4 * sizeof(unsigned long long));
  return e;
}

}  // namespace

namespace bfly_state {
bfly_status set_error(bfly_status s, const std::string &msg) { return fail(s, msg); }
}  // namespace bfly_state

namespace {
bfly_status autotune_create(bfly_plan_t *out, int dim, double N, int64_t nx, const double *x, int64_t nk,
                            const double *k, int p, bfly_opts o);
}

extern "C" {

const char *bfly_last_error(void) { return g_err.c_str(); }

const char *bfly_version(void) { return "bfly 0.2 sm_103a"; }

void bfly_plan_destroy(bfly_plan_t plan) {
  if (!plan) return;
  if (plan->dmem) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != plan->device) cudaSetDevice(plan->device);
    cudaFree(plan->dmem);
    if (cur != plan->device && cur >= 0) cudaSetDevice(cur);
  }
  delete plan;
}

bfly_status bfly_plan_create(bfly_plan_t *out, int dim, double N, int64_t nx, const double *x,
                             int64_t nk, const double *k, int p, const bfly_opts *opts) {
  g_err.clear();
  const auto t0 = std::chrono::steady_clock::now();
  if (!out) return fail(BFLY_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (dim != 2 && dim != 3) return fail(BFLY_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (p < 3 || p > 9) return fail(BFLY_ERR_INVALID_ARG, "p must be in 3..9");
  if (p % 2 == 0) return fail(BFLY_ERR_UNSUPPORTED, "the library has kernels for p = 3, 5, 7, 9");
  if (!std::isfinite(N) || !(N > 0)) return fail(BFLY_ERR_INVALID_ARG, "N must be finite and > 0");
  const int L = levels_for(N);
  if ((dim == 2 && L > 30) || (dim == 3 && L > 20))
    return fail(BFLY_ERR_UNSUPPORTED, "N too large for 64-bit Morton keys");
  if (nx < 0 || nk < 0 || nx > INT32_MAX / 2 || nk > INT32_MAX / 2)
    return fail(BFLY_ERR_INVALID_ARG, "nx and nk must be in [0, 2^30)");
  if ((nx > 0 && !x) || (nk > 0 && !k)) return fail(BFLY_ERR_INVALID_ARG, "x or k is NULL");
  bfly_opts o{};
  o.prec = BFLY_PREC_FP32;
  o.max_nrhs = 1;
  if (opts) o = *opts;
  if (o.prec != BFLY_PREC_FP32 && o.prec != BFLY_PREC_FP64 && o.prec != BFLY_PREC_TC)
    return fail(BFLY_ERR_INVALID_ARG, "unknown precision");
  if (o.prec == BFLY_PREC_TC && dim != 2)
    return fail(BFLY_ERR_UNSUPPORTED, "the tensor-core recursive step is built for dim = 2");
  // right-hand-side groups: the FP32 recursive step on groups of eight right-hand sides
  const bool rhs_groups = o.prec == BFLY_PREC_FP32 && (o.flags & BFLY_FLAG_RHS_GROUPS);
  if (rhs_groups && dim != 2)
    return fail(BFLY_ERR_UNSUPPORTED, "the right-hand-side grouped recursive step is built for dim = 2");
  if ((o.flags & BFLY_FLAG_DATAFLOW) && (o.prec == BFLY_PREC_TC || rhs_groups))
    return fail(BFLY_ERR_UNSUPPORTED, "the single-launch sweep runs the FP32 and FP64 recursive step");
  if (o.max_nrhs < 1 || o.max_nrhs > 4096) return fail(BFLY_ERR_INVALID_ARG, "max_nrhs must be in 1..4096");
  if (o.reserved != 0) return fail(BFLY_ERR_INVALID_ARG, "reserved options must be zero");
  if (o.stages < 0 || o.stages > bfly::kMaxLevels) return fail(BFLY_ERR_INVALID_ARG, "stages must be in 0..3");
  if ((o.flags & BFLY_FLAG_AUTOTUNE) && !(o.flags & BFLY_FLAG_HOST_ONLY))
    return autotune_create(out, dim, N, nx, x, nk, k, p, o);

  bfly_plan_t P = new (std::nothrow) bfly_plan_s();
  if (!P) return fail(BFLY_ERR_OUT_OF_MEMORY, "host allocation");
  P->dim = dim;
  P->p = p;
  P->L = L;
  P->N = N;
  P->rho = std::ldexp(N, -L);  // exact
  P->scale = P->rho == 1.0 ? 1.0 : std::sqrt(std::ldexp(1.0, L) / N);
  P->nx = nx;
  P->nk = nk;
  P->prec = o.prec;
  P->max_nrhs = o.max_nrhs;
  P->flags = o.flags;
  std::string err = bfly::build_tree(P->TX, dim, L, N, P->scale, nx, x);
  if (err.empty()) err = bfly::build_tree(P->TK, dim, L, N, P->scale, nk, k);
  if (!err.empty()) {
    delete P;
    return fail(BFLY_ERR_INVALID_ARG, err);
  }
  const int q = p - 1;
  int PD = 1;
  for (int d = 0; d < dim; ++d) PD *= p;
  P->elem_bytes = o.prec == BFLY_PREC_FP64 ? 16 : 8;
  // stage sizes: stage t pairs T_X level L-t with T_K level t
  P->pairs.resize(L + 1);
  int64_t maxp = 0, tot = 0;
  for (int t = 0; t <= L; ++t) {
    P->pairs[t] = P->TX.nbox(L - t) * P->TK.nbox(t);
    maxp = std::max(maxp, P->pairs[t]);
    tot += P->pairs[t];
  }
  bfly_plan_info_t &I = P->info;
  I.dim = dim;
  I.p = p;
  I.L = L;
  I.prec = o.prec;
  I.N = N;
  I.rho = P->rho;
  I.nx = nx;
  I.nk = nk;
  I.total_pairs = tot;
  I.max_pairs = maxp;
  for (int t = 0; t < L; ++t) {
    I.tiles_read_fwd += P->pairs[t + 1];
    I.tiles_written_fwd += P->pairs[t];
    I.jobs_fwd += P->TX.nbox(L - t) * P->TK.nbox(t + 1);
  }

  const bool host_only = (o.flags & BFLY_FLAG_HOST_ONLY) != 0;
  // shared memory plan of the recursive step
  P->ks = select_kernels(p, o.prec == BFLY_PREC_FP64 ? 0 : o.prec == BFLY_PREC_TC ? 2 : rhs_groups ? 3 : 1, dim);
  if (!P->ks) {
    delete P;
    return fail(BFLY_ERR_UNSUPPORTED, "no kernels for this (dim, p)");
  }
  size_t max_smem = 227 * 1024;
  if (!host_only) {
    int dev = 0, v = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) {
      delete P;
      return fail(BFLY_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
    }
    P->device = dev;
    max_smem = (size_t)v;
  }
  P->TS = P->ks->tile_stride;
  // capacities: the largest chunk that fits the shared-memory budget of one block
  // default budget: four blocks per SM in 2D; in 3D (8x larger tiles at p = 5) fewer,
  // larger blocks, whose chunks hold enough tiles to keep the consumer warps busy
  // (2D FP32: 72 KB, three blocks per SM, the autotuner's choice on the curve, star and
  // batched workloads; tensor-core step: eight right-hand sides per tile slot, two blocks
  // per SM)
  const int def_kb = (o.prec == BFLY_PREC_TC || rhs_groups) ? 110 : dim == 3 ? 73 : o.prec == BFLY_PREC_FP64 ? 55 : 72;
  const size_t want = (size_t)(o.smem_kb > 0 ? o.smem_kb : def_kb) * 1024;
  auto caps_for = [&](size_t budget) {
    // tile slots in steps of 8 (FP32, FP64); of 1 for the tensor-core step, whose slots hold
    // eight right-hand sides each
    const int step = (o.prec == BFLY_PREC_TC || rhs_groups) ? 1 : 8;
    for (int cap = 1024; cap >= step; cap -= step) {
      const ChunkCaps c{cap, cap, cap, P->ks->meta_bytes(cap, cap, cap)};
      if (P->ks->level_smem(c) <= budget) return c;
    }
    return ChunkCaps{0, 0, 0, 0};
  };
  ChunkCaps caps = caps_for(std::min(want, max_smem));
  if (caps.cap0 == 0) caps = caps_for(max_smem);
  if (caps.cap0 == 0) {
    delete P;
    return fail(BFLY_ERR_UNSUPPORTED, "charge tiles of this (dim, p, precision) do not fit in shared memory");
  }
  P->caps = caps;
  P->level_smem = P->ks->level_smem(caps);
  // the persistent grid of the recursive step (resident blocks per SM x SMs), for which
  // the stage programs are scheduled
  if (!host_only) {
    int blocks = 0, sms = 0;
    cudaError_t e = P->ks->level_setup(P->level_smem, &blocks);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) {
      delete P;
      return fail(BFLY_ERR_CUDA, std::string("recursive-step setup: ") + cudaGetErrorString(e));
    }
    if (blocks < 1) {
      const std::string msg = "recursive-step kernel cannot be resident with " +
                              std::to_string(P->level_smem) + " bytes of shared memory";
      delete P;
      return fail(BFLY_ERR_UNSUPPORTED, msg);
    }
    P->level_grid = blocks * sms;
    I.blocks_per_sm = blocks;
  }
  // steps of the sweep (forward order).  2D: three stages per launch, (2, 1, 0), (5, 4, 3),
  // ... from the bottom and the L mod 3 top stages together; a step whose units exceed the
  // shared-memory capacities gives up its last stage to a step of its own.  3D: one stage
  // per launch (a two-level unit holds up to 64 input tiles, more than a block's share of
  // shared memory)
  auto trees = [&](int t) {
    return bfly::StageTrees{&P->TX.cs[L - t - 1], &P->TX.idx[L - t], &P->TK.cs[t], &P->TK.idx[t + 1]};
  };
  std::deque<int> todo;
  // stages per launch: 2D up to three (default three); 3D up to two (default one: a 3D
  // two-level unit holds up to 64 input tiles of p^3 values, which only the sparse boxes
  // of surfaces keep within a block's shared memory)
  // (2D with BFLY_FLAG_DATAFLOW: two by default; the steps no longer cost a launch each, and
  // the smaller units of two stages measured faster in one launch: curve8192 0.192 against
  // 0.194 ms, star32768 0.749 against 0.766 ms)
  const int max_lev = (o.flags & BFLY_FLAG_ONE_STAGE) ? 1
                      : dim == 3 ? std::min(o.stages > 0 ? o.stages : 1, bfly::kMaxPasses / 3)
                      : o.stages > 0 ? o.stages
                      : (o.flags & BFLY_FLAG_DATAFLOW) ? 2 : bfly::kMaxLevels;
  if (max_lev == 1) {
    todo.assign(L, 1);
  } else {
    if (L % max_lev) todo.push_back(L % max_lev);
    for (int i = 0; i < L / max_lev; ++i) todo.push_back(max_lev);
  }
  I.stages_per_launch = max_lev;
  I.rhs_groups = rhs_groups ? 1 : 0;
  // the programs of the planned steps, forward and adjoint, compiled on all host cores
  // (each is independent); a step split after a capacity failure is compiled below
  struct Compiled {
    bfly::StageProgram prog;
    bool fits = true, used = false;
  };
  std::vector<std::pair<int, int>> groups;  // (t, levels)
  {
    int t = L - 1;
    for (int lev : todo) {
      groups.push_back({t, lev});
      t -= lev;
    }
  }
  std::vector<Compiled> pre(groups.size() * 2);
  std::atomic<int> compile_failed{0};  // 1: host memory exhausted, 2: another exception
  std::string compile_error;
  std::mutex compile_error_mutex;
  {
    std::atomic<size_t> next{0};
    auto worker = [&]() {
      for (size_t i; (i = next++) < pre.size();) {
        try {
          const int t = groups[i / 2].first, lev = groups[i / 2].second;
          bfly::StageTrees st[bfly::kMaxLevels];
          for (int l = 0; l < lev; ++l) st[l] = trees(t - l);
          pre[i].prog = bfly::make_step_program(dim, p, st, lev, (i & 1) != 0, caps, &pre[i].fits);
        } catch (const std::bad_alloc &) {
          compile_failed = 1;
        } catch (const std::exception &ex) {
          std::lock_guard<std::mutex> lock(compile_error_mutex);
          compile_failed = 2;
          compile_error = ex.what();
        } catch (...) {
          compile_failed = 2;
        }
      }
    };
    const size_t n_threads = std::min<size_t>(std::max(1u, std::thread::hardware_concurrency()), pre.size());
    std::vector<std::thread> threads;
    // threads that cannot be started leave their share to the others (the calling thread
    // at least)
    for (size_t i = 1; i < n_threads; ++i) {
      try {
        threads.emplace_back(worker);
      } catch (...) {
        break;
      }
    }
    worker();
    for (auto &th : threads) th.join();
  }
  if (compile_failed) {
    delete P;
    if (compile_failed == 1) return fail(BFLY_ERR_OUT_OF_MEMORY, "host memory exhausted while compiling the stage programs");
    return fail(BFLY_ERR_CUDA, "internal error while compiling the stage programs: " + compile_error);
  }
  auto compile = [&](int t, int lev, bool adjoint, bool *fits) {
    for (size_t g = 0; g < groups.size(); ++g)
      if (groups[g].first == t && groups[g].second == lev && !pre[2 * g + adjoint].used) {
        Compiled &c = pre[2 * g + adjoint];
        c.used = true;
        *fits = c.fits;
        return std::move(c.prog);
      }
    bfly::StageTrees st[bfly::kMaxLevels];
    for (int l = 0; l < lev; ++l) st[l] = trees(t - l);
    return bfly::make_step_program(dim, p, st, lev, adjoint, caps, fits);
  };
  std::vector<bfly_plan_s::Step> plan_steps;
  int64_t lanes_used_all = 0, lanes_issued_all = 0;
  for (int t = L - 1; !todo.empty();) {
    int lev = todo.front();
    todo.pop_front();
    bfly::StageProgram pf, pa;
    for (;;) {
      bool fits_f = true, fits_a = true;
      pf = compile(t, lev, false, &fits_f);
      pa = compile(t, lev, true, &fits_a);
      if ((fits_f && fits_a) || lev == 1) break;
      --lev;
      todo.push_front(1);
    }
    plan_steps.push_back({t, lev});
    const size_t si = plan_steps.size() - 1;
    const int t_lo = t - plan_steps[si].levels + 1;
    for (int dir = 0; dir < 2; ++dir) {
      const int64_t tin = dir ? P->pairs[t_lo] : P->pairs[t + 1], tout = dir ? P->pairs[t + 1] : P->pairs[t_lo];
      const std::string bad = bfly::validate_program(dir ? pa : pf, dim, p, caps, tin, tout);
      if (!bad.empty()) {
        delete P;
        return fail(BFLY_ERR_CUDA, "internal error in the stage program: " + bad);
      }
    }
    I.chunks_fwd += (int64_t)pf.chunks.size();
    int64_t srcs = 0;  // (output tile of a pass, source) pairs
    for (const auto &cd : pf.chunks) {
      const unsigned char *bp = pf.blob.data() + cd.blob_off;
      const int32_t *hdr = reinterpret_cast<const int32_t *>(bp);
      int64_t ni = 0;
      for (int j = 0; j < hdr[0]; ++j) ni += hdr[4 + j];
      const bfly::Item *it = reinterpret_cast<const bfly::Item *>(bp + bfly::kBlobHeader);
      for (int64_t i = 0; i < ni; ++i) srcs += 1 + (it[i].src1 != 0xffff);
      // lanes used by the steps of every pass (32 fibres per step, two-source fibres first)
      for (int j = 0; j < hdr[0]; ++j) {
        const int64_t nf = (int64_t)hdr[4 + j] * (PD / p), nf2 = (int64_t)hdr[4 + bfly::kMaxPasses + j] * (PD / p);
        lanes_used_all += nf + nf2;
        lanes_issued_all += ((nf + 31) / 32 + (nf2 + 31) / 32) * 32;
      }
    }
    // per source and fibre: p (p-1)/2 complex multiply-adds (8 flops) for the columns of
    // W off the parent nodes, (p+1)/2 complex additions (2 flops) for those on them
    double fib = 1.0;
    for (int d = 0; d < dim - 1; ++d) fib *= p;
    I.flops_fwd += (double)srcs * fib * (8.0 * p * (p - 1) / 2 + 2.0 * (p + 1) / 2);
    P->progF.push_back(std::move(pf));
    P->progA.push_back(std::move(pa));
    t -= lev;
  }
  P->steps = plan_steps;
  I.steps = (int)plan_steps.size();
  if ((o.flags & BFLY_FLAG_DATAFLOW) && !plan_steps.empty()) {
    if ((int64_t)I.chunks_fwd * o.max_nrhs >= INT32_MAX / 2) {
      delete P;
      return fail(BFLY_ERR_UNSUPPORTED, "the single-launch sweep numbers its items in 32 bits: fewer chunks x max_nrhs");
    }
    const std::string bad = build_flows(P);
    if (!bad.empty()) {
      delete P;
      return fail(BFLY_ERR_CUDA, "internal error in the single-launch sweep: " + bad);
    }
    P->dataflow = true;
    I.dataflow = 1;
  }
  I.lane_use_fwd = lanes_issued_all ? (double)lanes_used_all / (double)lanes_issued_all : 1.0;
  if (host_only) {
    I.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = P;
    return BFLY_OK;
  }

  // ---- device arrays
  std::vector<double> inv_den(p);
  for (int m = 0; m < p; ++m) {
    double den = 1.0;
    for (int n2 = 0; n2 < p; ++n2)
      if (n2 != m) den *= std::sin(M_PI * ((double)(m - n2) / ((double)q * q)));
    inv_den[m] = 1.0 / den;
  }
  std::vector<double> xs(x, x + nx * dim), kv(k, k + nk * dim);

  Arena A;
  A.add_vec(&P->perm_x, P->TX.perm);
  A.add_vec(&P->perm_k, P->TK.perm);
  A.add_vec(&P->leaf_x, P->TX.leaf_start);
  A.add_vec(&P->leaf_k, P->TK.leaf_start);
  A.add_vec(&P->pleaf_x, P->TX.point_leaf);
  A.add_vec(&P->pleaf_k, P->TK.point_leaf);
  A.add_vec(&P->off_x, P->TX.off);
  A.add_vec(&P->off_k, P->TK.off);
  A.add_vec(&P->xs, xs);
  A.add_vec(&P->ks_, kv);
  A.add_vec(&P->inv_den, inv_den);
  A.add(&P->Wx, (size_t)nx * dim * p * P->elem_bytes);
  A.add(&P->Wk, (size_t)nk * dim * p * P->elem_bytes);
  const size_t n_steps = P->steps.size();
  P->dF.resize(n_steps);
  P->dA.resize(n_steps);
  for (size_t si = 0; si < n_steps; ++si) {
    for (int dir = 0; dir < 2; ++dir) {
      StageProgram &pg = dir ? P->progA[si] : P->progF[si];
      bfly_plan_s::DevProg &dp = dir ? P->dA[si] : P->dF[si];
      A.add_vec(&dp.chunks, pg.chunks);
      A.add_vec(&dp.blob, pg.blob);
      A.add_vec(&dp.runs, pg.runs);
    }
  }
  static const int zero_status = 0;
  A.add(reinterpret_cast<void **>(&P->status), sizeof(int), &zero_status);
  const std::vector<unsigned long long> zero_sched((size_t)4 * std::max<size_t>(n_steps, 1), 0ull);
  A.add_vec(&P->sched, zero_sched);
  const size_t buf_bytes = (size_t)maxp * P->TS * P->elem_bytes * o.max_nrhs;
  A.add(&P->buf[0], buf_bytes);
  A.add(&P->buf[1], buf_bytes);
  const size_t stage_bytes = (size_t)std::max(nx, nk) * 16 * o.max_nrhs;
  A.add(&P->stage_in, stage_bytes);
  A.add(&P->stage_out, stage_bytes);
  if (P->dataflow) {
    // a buffer per inner boundary of the sweep (boundary b: the last stage of step b - 1)
    P->fbuf.assign(n_steps + 1, nullptr);
    for (size_t b = 1; b < n_steps; ++b) {
      const bfly_plan_s::Step &st = P->steps[b - 1];
      A.add(&P->fbuf[b], (size_t)P->pairs[st.t - st.levels + 1] * P->TS * P->elem_bytes * o.max_nrhs);
    }
    for (bfly_plan_s::Flow *F : {&P->flowF, &P->flowA}) {
      A.add(reinterpret_cast<void **>(&F->entries), (size_t)F->n_entries * sizeof(bfly::BatchEntry));
      A.add_vec(&F->deps_d, F->deps);
      A.add_vec(&F->dep_off_d, F->dep_off);
      A.add_vec(&F->dep_idx_d, F->dep_idx);
      A.add_vec(&F->first_use_d, F->first_use);
      A.add(reinterpret_cast<void **>(&F->flags), (size_t)F->n_entries * o.max_nrhs * sizeof(unsigned));
    }
    A.add(reinterpret_cast<void **>(&P->epoch), 2 * sizeof(unsigned));
    A.add(reinterpret_cast<void **>(&P->flow_sched), 4 * sizeof(unsigned long long));
  }

  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&P->dmem), A.total);
  if (e != cudaSuccess) {
    delete P;
    return fail(e == cudaErrorMemoryAllocation ? BFLY_ERR_OUT_OF_MEMORY : BFLY_ERR_CUDA,
                std::string("cudaMalloc of the plan: ") + cudaGetErrorString(e));
  }
  P->dbytes = A.total;
  size_t at = 0;
  for (auto &it : A.items) {
    *it.slot = P->dmem + at;
    if (it.host && it.bytes) {
      e = cudaMemcpy(*it.slot, it.host, it.bytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) break;
    }
    at += (it.bytes + 255) & ~(size_t)255;
  }
  if (e == cudaSuccess && P->dataflow) e = upload_flows(P);
  if (e == cudaSuccess)
    e = bfly::launch_weights(o.prec == BFLY_PREC_FP64 ? 0 : 1, nk, dim, p, 0, P->off_k, P->inv_den, P->Wk, 0);
  if (e == cudaSuccess)
    e = bfly::launch_weights(o.prec == BFLY_PREC_FP64 ? 0 : 1, nx, dim, p, 1, P->off_x, P->inv_den, P->Wx, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    const std::string msg = std::string("plan upload: ") + cudaGetErrorString(e);
    bfly_plan_destroy(P);
    return fail(BFLY_ERR_CUDA, msg);
  }
  I.smem_kb = (int)((P->level_smem + 1023) / 1024);
  I.workspace_bytes = (int64_t)P->dbytes;
  I.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = P;
  return BFLY_OK;
}

}  // extern "C"

namespace {

bfly_status check_exec(bfly_plan_t P, const void *a, const void *b, int nrhs, int dtype, bool adjoint) {
  if (!P) return fail(BFLY_ERR_INVALID_ARG, "plan is NULL");
  if (!P->dmem) return fail(BFLY_ERR_INVALID_ARG, "plan was created host-only");
  // a pointer may be NULL only when its side has no points
  const int64_t n_a = adjoint ? P->nx : P->nk, n_b = adjoint ? P->nk : P->nx;
  if ((!a && n_a > 0) || (!b && n_b > 0)) return fail(BFLY_ERR_INVALID_ARG, "data pointer is NULL");
  if (nrhs < 1 || nrhs > P->max_nrhs) return fail(BFLY_ERR_INVALID_ARG, "nrhs outside 1..max_nrhs");
  if (dtype != BFLY_C64 && dtype != BFLY_C128) return fail(BFLY_ERR_INVALID_ARG, "unknown dtype");
  return BFLY_OK;
}

// Launches the sweep on stream s; when ev is non-null, records ev[i] before launch i and
// ev[steps + 2] after the last one.
bfly_status run(bfly_plan_t P, const void *in, void *out, int nrhs, int dtype, bool adjoint,
                cudaStream_t s, cudaEvent_t const *ev = nullptr) {
  const bool io64 = dtype == BFLY_C128;
  const int L = P->L, PD = P->TS, S = (int)P->steps.size();
  int n = 0;
  auto mark = [&]() -> cudaError_t {
    cudaEvent_t e = ev ? ev[n++] : nullptr;
    return e ? cudaEventRecord(e, s) : cudaSuccess;
  };
  // an empty side: nothing to compute (no outputs) or every output is zero (no inputs)
  const int64_t n_in = adjoint ? P->nx : P->nk, n_out = adjoint ? P->nk : P->nx;
  if (n_in == 0 || n_out == 0) {
    BFLY_CUDA(mark());
    if (n_out > 0) BFLY_CUDA(cudaMemsetAsync(out, 0, (size_t)nrhs * n_out * (io64 ? 16 : 8), s));
    while (ev && n < S + 3) BFLY_CUDA(mark());
    return BFLY_OK;
  }
  if (!adjoint) {
    // step 2: leaf charges (stage L) from the sources
    BFLY_CUDA(mark());
    BFLY_CUDA(P->ks->spread(point_args(P, false, in, P->buf[0], nrhs, io64, false,
                                       P->pairs[L] * PD), s));
    // step 3: stages L-1 .. 0, up to three per launch, or all in one launch
    if (P->dataflow) {
      BFLY_CUDA(mark());
      BFLY_CUDA(P->ks->level(flow_args(P, false, nrhs), false, P->level_grid, P->level_smem, s));
      for (int si = 1; si < S; ++si) BFLY_CUDA(mark());
    } else {
      for (int si = 0; si < S; ++si) {
        BFLY_CUDA(mark());
        BFLY_CUDA(P->ks->level(level_args(P, si, false, nrhs), false, P->level_grid, P->level_smem, s));
      }
    }
    // step 4: evaluate at the targets from stage 0
    BFLY_CUDA(mark());
    BFLY_CUDA(P->ks->interp(point_args(P, true, P->buf[P->dataflow ? 1 : S & 1], out, nrhs, io64, false,
                                       P->pairs[0] * PD), s));
  } else {
    BFLY_CUDA(mark());
    BFLY_CUDA(P->ks->spread(point_args(P, true, in, P->buf[P->dataflow ? 1 : S & 1], nrhs, io64, true,
                                       P->pairs[0] * PD), s));
    if (P->dataflow) {
      BFLY_CUDA(mark());
      BFLY_CUDA(P->ks->level(flow_args(P, true, nrhs), true, P->level_grid, P->level_smem, s));
      for (int si = 1; si < S; ++si) BFLY_CUDA(mark());
    } else {
      for (int si = S - 1; si >= 0; --si) {
        BFLY_CUDA(mark());
        BFLY_CUDA(P->ks->level(level_args(P, si, true, nrhs), true, P->level_grid, P->level_smem, s));
      }
    }
    BFLY_CUDA(mark());
    BFLY_CUDA(P->ks->interp(point_args(P, false, P->buf[0], out, nrhs, io64, true,
                                       P->pairs[L] * PD), s));
  }
  BFLY_CUDA(mark());
  return BFLY_OK;
}

}  // namespace

extern "C" {

bfly_status bfly_execute(bfly_plan_t plan, const void *f, void *u, int nrhs, int dtype, void *stream) {
  g_err.clear();
  bfly_status st = check_exec(plan, f, u, nrhs, dtype, false);
  if (st != BFLY_OK) return st;
  return run(plan, f, u, nrhs, dtype, false, reinterpret_cast<cudaStream_t>(stream));
}

bfly_status bfly_execute_adjoint(bfly_plan_t plan, const void *u, void *f, int nrhs, int dtype,
                                 void *stream) {
  g_err.clear();
  bfly_status st = check_exec(plan, u, f, nrhs, dtype, true);
  if (st != BFLY_OK) return st;
  return run(plan, u, f, nrhs, dtype, true, reinterpret_cast<cudaStream_t>(stream));
}

bfly_status bfly_execute_host(bfly_plan_t plan, const void *in_host, void *out_host, int nrhs,
                              int dtype, int adjoint, void *stream) {
  g_err.clear();
  bfly_status st = check_exec(plan, in_host, out_host, nrhs, dtype, adjoint != 0);
  if (st != BFLY_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t eb = dtype == BFLY_C128 ? 16 : 8;
  const int64_t nin = adjoint ? plan->nx : plan->nk, nout = adjoint ? plan->nk : plan->nx;
  // Pinned host buffers are addressable from the device: the leaf step then gathers the
  // input straight from host memory and the final step scatters the result into it,
  // with no staging copies.  Other (pageable) buffers go through the plan's device
  // staging buffers.
  if (nin > 0 && nout > 0) {
    cudaPointerAttributes ai{}, ao{};
    if (cudaPointerGetAttributes(&ai, in_host) == cudaSuccess && cudaPointerGetAttributes(&ao, out_host) == cudaSuccess &&
        ai.type == cudaMemoryTypeHost && ao.type == cudaMemoryTypeHost && ai.devicePointer && ao.devicePointer) {
      st = run(plan, ai.devicePointer, ao.devicePointer, nrhs, dtype, adjoint != 0, s);
      if (st != BFLY_OK) return st;
      BFLY_CUDA(cudaStreamSynchronize(s));
      return BFLY_OK;
    }
    cudaGetLastError();  // a pageable pointer is not an error
  }
  if (nin > 0)
    BFLY_CUDA(cudaMemcpyAsync(plan->stage_in, in_host, (size_t)nin * nrhs * eb, cudaMemcpyHostToDevice, s));
  st = run(plan, plan->stage_in, plan->stage_out, nrhs, dtype, adjoint != 0, s);
  if (st != BFLY_OK) return st;
  if (nout > 0)
    BFLY_CUDA(cudaMemcpyAsync(out_host, plan->stage_out, (size_t)nout * nrhs * eb, cudaMemcpyDeviceToHost, s));
  BFLY_CUDA(cudaStreamSynchronize(s));
  return BFLY_OK;
}

bfly_status bfly_execute_events(bfly_plan_t plan, const void *in, void *out, int nrhs, int dtype,
                                int adjoint, void *stream, void *const *events, int n_events) {
  g_err.clear();
  bfly_status st = check_exec(plan, in, out, nrhs, dtype, adjoint != 0);
  if (st != BFLY_OK) return st;
  if (!events || n_events != (int)plan->steps.size() + 3)
    return fail(BFLY_ERR_INVALID_ARG, "events must hold steps + 3 entries (bfly_plan_info_t.steps)");
  return run(plan, in, out, nrhs, dtype, adjoint != 0, reinterpret_cast<cudaStream_t>(stream),
             reinterpret_cast<cudaEvent_t const *>(events));
}

}  // extern "C"

namespace {

// The boundary b of the plan's launches (0: stage L; s + 1: after recursive-step launch s)
// holding stage t, or -1 when no launch ends at stage t.
int boundary_of(bfly_plan_t P, int t) {
  if (t == P->L) return 0;
  for (size_t s = 0; s < P->steps.size(); ++s)
    if (P->steps[s].t - P->steps[s].levels + 1 == t) return (int)s + 1;
  return -1;
}

// Arguments of the split sweep: a device plan, the point-side pointer (NULL only when
// that side has no points), nrhs and dtype.
bfly_status check_split(bfly_plan_t P, const void *v, int64_t n, int nrhs, int dtype) {
  if (!P) return fail(BFLY_ERR_INVALID_ARG, "plan is NULL");
  if (!P->dmem) return fail(BFLY_ERR_INVALID_ARG, "plan was created host-only");
  if (!v && n > 0) return fail(BFLY_ERR_INVALID_ARG, "data pointer is NULL");
  if (nrhs < 1 || nrhs > P->max_nrhs) return fail(BFLY_ERR_INVALID_ARG, "nrhs outside 1..max_nrhs");
  if (dtype != BFLY_C64 && dtype != BFLY_C128) return fail(BFLY_ERR_INVALID_ARG, "unknown dtype");
  return BFLY_OK;
}

bfly_status check_stage(bfly_plan_t P, int t, const void *charges, int *b) {
  if (t < 0 || t > P->L) return fail(BFLY_ERR_INVALID_ARG, "stage outside 0..L");
  *b = boundary_of(P, t);
  if (*b < 0)
    return fail(BFLY_ERR_INVALID_ARG, "stage " + std::to_string(t) +
                                          " is not at a launch boundary of the plan (bfly_plan_step; "
                                          "stages = 1 makes every stage one)");
  if (!charges && P->pairs[t] > 0) return fail(BFLY_ERR_INVALID_ARG, "charges pointer is NULL");
  return BFLY_OK;
}

}  // namespace

extern "C" {

bfly_status bfly_execute_to_stage(bfly_plan_t plan, const void *in, int t, void *charges, int nrhs, int dtype,
                                  int adjoint, void *stream) {
  g_err.clear();
  bfly_status st = check_split(plan, in, plan ? (adjoint ? plan->nx : plan->nk) : 0, nrhs, dtype);
  if (st != BFLY_OK) return st;
  int b = 0;
  st = check_stage(plan, t, charges, &b);
  if (st != BFLY_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool io64 = dtype == BFLY_C128;
  const size_t bytes = (size_t)nrhs * plan->pairs[t] * plan->TS * plan->elem_bytes;
  const int L = plan->L, S = (int)plan->steps.size();
  if (plan->nk == 0 || plan->nx == 0) {  // an empty side: zero charges, or no tiles at all
    if (bytes) BFLY_CUDA(cudaMemsetAsync(charges, 0, bytes, s));
    return BFLY_OK;
  }
  if (!adjoint) {
    // leaf step, then the launches from boundary 0 (stage L) to boundary b (stage t)
    BFLY_CUDA(plan->ks->spread(point_args(plan, false, in, plan->buf[0], nrhs, io64, false,
                                          plan->pairs[L] * plan->TS), s));
    for (int si = 0; si < b; ++si)
      BFLY_CUDA(plan->ks->level(level_args(plan, si, false, nrhs), false, plan->level_grid, plan->level_smem, s));
  } else {
    // the final step's transpose, then the adjoint launches from boundary S (stage 0) back
    // to boundary b (stage t)
    BFLY_CUDA(plan->ks->spread(point_args(plan, true, in, plan->buf[S & 1], nrhs, io64, true,
                                          plan->pairs[0] * plan->TS), s));
    for (int si = S - 1; si >= b; --si)
      BFLY_CUDA(plan->ks->level(level_args(plan, si, true, nrhs), true, plan->level_grid, plan->level_smem, s));
  }
  if (bytes) BFLY_CUDA(cudaMemcpyAsync(charges, plan->buf[b & 1], bytes, cudaMemcpyDeviceToDevice, s));
  return BFLY_OK;
}

bfly_status bfly_execute_from_stage(bfly_plan_t plan, const void *charges, int t, void *out, int nrhs, int dtype,
                                    int adjoint, void *stream) {
  g_err.clear();
  const int64_t n_out = plan ? (adjoint ? plan->nk : plan->nx) : 0, n_in = plan ? (adjoint ? plan->nx : plan->nk) : 0;
  bfly_status st = check_split(plan, out, n_out, nrhs, dtype);
  if (st != BFLY_OK) return st;
  int b = 0;
  st = check_stage(plan, t, charges, &b);
  if (st != BFLY_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool io64 = dtype == BFLY_C128;
  const int L = plan->L, S = (int)plan->steps.size();
  if (n_out == 0) return BFLY_OK;
  if (n_in == 0) {
    BFLY_CUDA(cudaMemsetAsync(out, 0, (size_t)nrhs * n_out * (io64 ? 16 : 8), s));
    return BFLY_OK;
  }
  const size_t bytes = (size_t)nrhs * plan->pairs[t] * plan->TS * plan->elem_bytes;
  if (bytes) BFLY_CUDA(cudaMemcpyAsync(plan->buf[b & 1], charges, bytes, cudaMemcpyDeviceToDevice, s));
  if (!adjoint) {
    // the launches from boundary b to boundary S (stage 0), then the final step
    for (int si = b; si < S; ++si)
      BFLY_CUDA(plan->ks->level(level_args(plan, si, false, nrhs), false, plan->level_grid, plan->level_smem, s));
    BFLY_CUDA(plan->ks->interp(point_args(plan, true, plan->buf[S & 1], out, nrhs, io64, false,
                                          plan->pairs[0] * plan->TS), s));
  } else {
    // the adjoint launches from boundary b back to boundary 0 (stage L), then the leaf
    // step's transpose
    for (int si = b - 1; si >= 0; --si)
      BFLY_CUDA(plan->ks->level(level_args(plan, si, true, nrhs), true, plan->level_grid, plan->level_smem, s));
    BFLY_CUDA(plan->ks->interp(point_args(plan, false, plan->buf[0], out, nrhs, io64, true,
                                          plan->pairs[L] * plan->TS), s));
  }
  return BFLY_OK;
}

bfly_status bfly_direct(bfly_plan_t plan, const void *in, void *out, int nrhs, int dtype, int adjoint,
                        void *stream) {
  g_err.clear();
  bfly_status st = check_exec(plan, in, out, nrhs, dtype, adjoint != 0);
  if (st != BFLY_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int prec = plan->prec == BFLY_PREC_FP64 ? 0 : 1;
  if (!adjoint)
    BFLY_CUDA(bfly::launch_direct(prec, plan->dim, plan->N, plan->nx, plan->xs, plan->nk, plan->ks_,
                                  in, out, nrhs, dtype == BFLY_C128, +1.0, s));
  else
    BFLY_CUDA(bfly::launch_direct(prec, plan->dim, plan->N, plan->nk, plan->ks_, plan->nx, plan->xs,
                                  in, out, nrhs, dtype == BFLY_C128, -1.0, s));
  return BFLY_OK;
}

bfly_status bfly_device_status(bfly_plan_t plan, int *flags) {
  g_err.clear();
  if (!plan || !plan->status) return fail(BFLY_ERR_INVALID_ARG, "plan is NULL or host-only");
  int v = 0;
  BFLY_CUDA(cudaDeviceSynchronize());
  BFLY_CUDA(cudaMemcpy(&v, plan->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) BFLY_CUDA(cudaMemset(plan->status, 0, sizeof(int)));
  if (flags) *flags = v;
  if (v) return fail(BFLY_ERR_TIMEOUT, "a bounded device-side wait gave up (status bits " + std::to_string(v) + ")");
  return BFLY_OK;
}

bfly_status bfly_stream_status(bfly_plan_t plan, void *stream, int *flags) {
  g_err.clear();
  if (!plan || !plan->status) return fail(BFLY_ERR_INVALID_ARG, "plan is NULL or host-only");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int v = 0;
  // a copy to pageable memory returns once it has completed, after the stream's earlier work
  BFLY_CUDA(cudaMemcpyAsync(&v, plan->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  BFLY_CUDA(cudaStreamSynchronize(s));
  if (v) BFLY_CUDA(cudaMemsetAsync(plan->status, 0, sizeof(int), s));
  if (flags) *flags = v;
  if (v) return fail(BFLY_ERR_TIMEOUT, "a bounded device-side wait gave up (status bits " + std::to_string(v) + ")");
  return BFLY_OK;
}

bfly_status bfly_plan_info(bfly_plan_t plan, bfly_plan_info_t *info) {
  if (!plan || !info) return fail(BFLY_ERR_INVALID_ARG, "plan or info is NULL");
  *info = plan->info;
  return BFLY_OK;
}

bfly_status bfly_plan_step(bfly_plan_t plan, int s, int *t, int *levels) {
  if (!plan || !t || !levels) return fail(BFLY_ERR_INVALID_ARG, "NULL argument");
  if (s < 0 || s >= (int)plan->steps.size()) return fail(BFLY_ERR_INVALID_ARG, "step outside 0..steps-1");
  *t = plan->steps[s].t;
  *levels = plan->steps[s].levels;
  return BFLY_OK;
}

bfly_status bfly_plan_program(bfly_plan_t plan, int s, int adjoint, int what, void *out, int64_t cap,
                              int64_t *bytes) {
  if (!plan || !bytes) return fail(BFLY_ERR_INVALID_ARG, "NULL argument");
  if (s < 0 || s >= (int)plan->steps.size()) return fail(BFLY_ERR_INVALID_ARG, "step outside 0..steps-1");
  if (what < 0 || what > 2) return fail(BFLY_ERR_INVALID_ARG, "what must be 0, 1 or 2");
  const bfly::StageProgram &pg = adjoint ? plan->progA[s] : plan->progF[s];
  const void *src = what == 0 ? (const void *)pg.chunks.data() : what == 1 ? (const void *)pg.blob.data()
                                                                            : (const void *)pg.runs.data();
  const int64_t n = what == 0 ? (int64_t)(pg.chunks.size() * sizeof(bfly::ChunkDesc))
                    : what == 1 ? (int64_t)pg.blob.size()
                                : (int64_t)(pg.runs.size() * sizeof(bfly::Run));
  *bytes = n;
  if (out && cap > 0 && n > 0) std::memcpy(out, src, (size_t)std::min(n, cap));
  return BFLY_OK;
}

bfly_status bfly_plan_boxes(bfly_plan_t plan, int side, int lev, int32_t *out, int64_t cap, int64_t *n) {
  if (!plan || !n) return fail(BFLY_ERR_INVALID_ARG, "NULL argument");
  if (side < 0 || side > 1 || lev < 0 || lev > plan->L) return fail(BFLY_ERR_INVALID_ARG, "side or level out of range");
  const bfly::HostTree &T = side ? plan->TK : plan->TX;
  *n = T.nbox(lev);
  if (out && cap > 0) std::memcpy(out, T.idx[lev].data(), (size_t)std::min(*n, cap) * plan->dim * sizeof(int32_t));
  return BFLY_OK;
}

bfly_status bfly_plan_stage(bfly_plan_t plan, int t, int64_t *nA, int64_t *nB) {
  if (!plan || !nA || !nB) return fail(BFLY_ERR_INVALID_ARG, "NULL argument");
  if (t < 0 || t > plan->L) return fail(BFLY_ERR_INVALID_ARG, "stage outside 0..L");
  *nA = plan->TX.nbox(plan->L - t);
  *nB = plan->TK.nbox(t);
  return BFLY_OK;
}

}  // extern "C"

namespace {

// ---- autotuning of the recursive step (BFLY_FLAG_AUTOTUNE)

std::string tune_key(int dim, int p, int prec, int nrhs, int64_t max_pairs) {
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::string name = prop.name;
  for (auto &ch : name)
    if (ch == ' ') ch = '_';
  int size_class = 0;  // log2 of the largest stage's pair count
  while ((int64_t(1) << (size_class + 1)) <= max_pairs) ++size_class;
  return name + " d" + std::to_string(dim) + " p" + std::to_string(p) + " prec" + std::to_string(prec) +
         " nrhs" + std::to_string(nrhs) + " pairs2^" + std::to_string(size_class);
}

// One configuration of the recursive step: shared-memory budget per block, stages per
// launch (2D), precision of the applies.
struct TuneChoice {
  int smem_kb = 0, stages = 0, prec = -1, groups = 0;  // groups: BFLY_FLAG_RHS_GROUPS
  int flow = -1;  // BFLY_FLAG_DATAFLOW: 1 on, 0 off, -1 as requested
};

// The last choice recorded for `key` ("<key> <smem_kb> [<stages> <prec> [<groups>
// [<flow>]]]" lines), or smem_kb = 0 when there is none.
TuneChoice cache_lookup(const char *path, const std::string &key) {
  TuneChoice found;
  if (!path) return found;
  FILE *fh = std::fopen(path, "r");
  if (!fh) return found;
  char line[512];
  while (std::fgets(line, sizeof line, fh)) {
    std::string l(line);
    if (l.compare(0, key.size(), key) != 0 || l.size() <= key.size() || l[key.size()] != ' ') continue;
    TuneChoice c;
    const int n = std::sscanf(l.c_str() + key.size(), " %d %d %d %d %d", &c.smem_kb, &c.stages, &c.prec, &c.groups,
                              &c.flow);
    if (n >= 1 && c.smem_kb > 0) {
      if (n < 3) c.stages = 0, c.prec = -1;
      if (n < 4) c.groups = 0;
      if (n < 5) c.flow = -1;
      found = c;
    }
  }
  std::fclose(fh);
  return found;
}

void cache_store(const char *path, const std::string &key, const TuneChoice &c) {
  if (!path) return;
  FILE *fh = std::fopen(path, "a");
  if (!fh) return;
  std::fprintf(fh, "%s %d %d %d %d %d\n", key.c_str(), c.smem_kb, c.stages, c.prec, c.groups, c.flow);
  std::fclose(fh);
}

// Time of one forward sweep (median of 3 after a warm-up) on the plan's staging buffers.
bfly_status time_plan(bfly_plan_t P, double *ms) {
  const int nrhs = P->max_nrhs;
  const size_t bytes = (size_t)std::max(P->nx, P->nk) * 16 * nrhs;
  BFLY_CUDA(cudaMemset(P->stage_in, 0, bytes));
  cudaEvent_t e0, e1;
  BFLY_CUDA(cudaEventCreate(&e0));
  BFLY_CUDA(cudaEventCreate(&e1));
  std::vector<float> t;
  bfly_status st = BFLY_OK;
  for (int r = 0; r < 4 && st == BFLY_OK; ++r) {
    cudaEventRecord(e0, 0);
    st = run(P, P->stage_in, P->stage_out, nrhs, BFLY_C64, false, 0);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float v = 0;
    cudaEventElapsedTime(&v, e0, e1);
    if (r > 0) t.push_back(v);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BFLY_OK) return st;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return BFLY_OK;
}

bfly_status autotune_create(bfly_plan_t *out, int dim, double N, int64_t nx, const double *x, int64_t nk,
                            const double *k, int p, bfly_opts o) {
  o.flags &= ~BFLY_FLAG_AUTOTUNE;
  // a host-only plan first: the size class of the key
  bfly_opts ho = o;
  ho.flags |= BFLY_FLAG_HOST_ONLY;
  bfly_plan_t H = nullptr;
  bfly_status st = bfly_plan_create(&H, dim, N, nx, x, nk, k, p, &ho);
  if (st != BFLY_OK) return st;
  const std::string key = tune_key(dim, p, o.prec, o.max_nrhs, H->info.max_pairs);
  bfly_plan_destroy(H);
  auto with = [&](const TuneChoice &c) {
    bfly_opts r = o;
    r.smem_kb = c.smem_kb;
    if (c.stages > 0) r.stages = c.stages;
    if (c.prec >= 0) r.prec = c.prec;
    if (c.groups) r.flags |= BFLY_FLAG_RHS_GROUPS;
    else r.flags &= ~BFLY_FLAG_RHS_GROUPS;
    if (c.flow == 1) r.flags |= BFLY_FLAG_DATAFLOW;
    if (c.flow == 0) r.flags &= ~BFLY_FLAG_DATAFLOW;
    // the single-launch sweep runs the FP32 and FP64 kernels only
    if (c.groups || r.prec == BFLY_PREC_TC) r.flags &= ~BFLY_FLAG_DATAFLOW;
    return r;
  };
  const TuneChoice cached = cache_lookup(o.tune_cache, key);
  if (cached.smem_kb > 0) {
    const bfly_opts r = with(cached);
    return bfly_plan_create(out, dim, N, nx, x, nk, k, p, &r);
  }
  // candidates: budgets x stages per launch (2D); the tensor-core step for FP32 plans in
  // 2D with at least eight right-hand sides
  std::vector<TuneChoice> cands;
  const bool fixed_stages = o.stages > 0 || (o.flags & BFLY_FLAG_ONE_STAGE);
  if (dim == 2) {
    for (int stg : {3, 2, 1}) {
      if (fixed_stages && stg != (o.stages > 0 ? o.stages : 1)) continue;
      for (int kb : {40, 55, 73, 110}) cands.push_back({kb, stg, o.prec});
    }
    if (o.prec == BFLY_PREC_FP32 && o.max_nrhs >= 4)
      for (int stg : {3, 2}) {
        if (fixed_stages && stg != (o.stages > 0 ? o.stages : 1)) continue;
        for (int kb : {110, 220}) cands.push_back({kb, stg, BFLY_PREC_FP32, 1});
      }
    if (o.prec == BFLY_PREC_FP32 && o.max_nrhs >= 8)
      for (int stg : {3, 1}) {
        if (fixed_stages && stg != (o.stages > 0 ? o.stages : 1)) continue;
        for (int kb : {110, 220}) cands.push_back({kb, stg, BFLY_PREC_TC});
      }
  } else {
    // 3D: one stage per launch unless asked (the units of two stages of surfaces exceed a
    // block's shared memory, and the plan then falls back to one stage anyway)
    for (int kb : {40, 55, 73, 110, 220}) cands.push_back({kb, 0, o.prec});
  }
  bfly_plan_t best = nullptr;
  double best_ms = 0;
  TuneChoice best_c;
  for (const TuneChoice &c : cands) {
    const bfly_opts r = with(c);
    bfly_plan_t P = nullptr;
    if (bfly_plan_create(&P, dim, N, nx, x, nk, k, p, &r) != BFLY_OK) continue;
    double ms = 0;
    if (time_plan(P, &ms) != BFLY_OK) {
      bfly_plan_destroy(P);
      continue;
    }
    if (!best || ms < best_ms) {
      if (best) bfly_plan_destroy(best);
      best = P;
      best_ms = ms;
      best_c = c;
    } else {
      bfly_plan_destroy(P);
    }
  }
  if (!best) return fail(BFLY_ERR_UNSUPPORTED, "autotuning: no candidate configuration could be built");
  // the best FP32 / FP64 configuration with the single-launch sweep switched the other way
  // (switched on in 2D: at two and three stages per step, unless the stages were given)
  best_c.flow = best->dataflow ? 1 : 0;
  if (best->prec != BFLY_PREC_TC && !best_c.groups) {
    std::vector<TuneChoice> flips;
    TuneChoice c = best_c;
    c.flow = 1 - best_c.flow;
    if (c.flow == 1 && dim == 2 && !fixed_stages) {
      for (int stg : {2, 3}) {
        c.stages = stg;
        flips.push_back(c);
      }
    } else {
      flips.push_back(c);
    }
    for (const TuneChoice &f : flips) {
      const bfly_opts r = with(f);
      bfly_plan_t P = nullptr;
      double ms = 0;
      if (bfly_plan_create(&P, dim, N, nx, x, nk, k, p, &r) != BFLY_OK) continue;
      if (time_plan(P, &ms) == BFLY_OK && ms < best_ms) {
        bfly_plan_destroy(best);
        best = P;
        best_ms = ms;
        best_c = f;
      } else {
        bfly_plan_destroy(P);
      }
    }
  }
  best->info.tuned_ms = best_ms;
  cache_store(o.tune_cache, key, best_c);
  g_err.clear();
  *out = best;
  return BFLY_OK;
}

}  // namespace
