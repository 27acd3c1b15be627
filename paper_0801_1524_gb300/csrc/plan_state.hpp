// Internal state of a plan and the argument blocks of its kernels, shared by the
// translation units of the C ABI (api.cu, noalloc.cu).
#pragma once

#include <string>
#include <vector>

#include "../../include/bfly.h"
#include "kernels.hpp"
#include "plan.hpp"

struct bfly_plan_s {
  int dim = 0, p = 0, L = 0, prec = 1, max_nrhs = 1;
  unsigned flags = 0;
  double N = 0, rho = 1.0;  // rho = N / 2^L
  double scale = 1.0;       // points are scaled by sqrt(2^L / N) (1 when N = 2^L)
  int64_t nx = 0, nk = 0;
  int device = -1;
  bfly::HostTree TX, TK;
  const bfly::KernelSet *ks = nullptr;
  bfly::ChunkCaps caps{};
  int level_grid = 0, TS = 0;
  size_t level_smem = 0, elem_bytes = 0;
  // steps of the recursive step in forward order: stages t .. t - levels + 1 in one launch
  struct Step {
    int t, levels;
  };
  std::vector<Step> steps;
  std::vector<bfly::StageProgram> progF, progA;  // per step
  std::vector<int64_t> pairs;              // per stage t in [0, L]
  // device memory: one allocation carved into the arrays below
  char *dmem = nullptr;
  size_t dbytes = 0;
  int32_t *perm_x = nullptr, *perm_k = nullptr, *leaf_x = nullptr, *leaf_k = nullptr;
  int32_t *pleaf_x = nullptr, *pleaf_k = nullptr;
  double *off_x = nullptr, *off_k = nullptr, *xs = nullptr, *ks_ = nullptr, *inv_den = nullptr;
  void *Wx = nullptr, *Wk = nullptr;
  struct DevProg {
    bfly::ChunkDesc *chunks = nullptr;
    unsigned char *blob = nullptr;
    bfly::Run *runs = nullptr;
  };
  int *status = nullptr;  // device status word (bfly_device_status)
  // work counters of the recursive-step launches, [direction][stage t][2] (LevelArgs::sched)
  unsigned long long *sched = nullptr;
  std::vector<DevProg> dF, dA;  // per step
  // stage buffers: the charges between steps; boundary b (b = 0: stage L, b = s + 1: after
  // forward step s, b = steps: stage 0) lives in buf[b mod 2]
  void *buf[2] = {nullptr, nullptr};
  void *stage_in = nullptr, *stage_out = nullptr;
  // single-launch sweep (BFLY_FLAG_DATAFLOW), per direction: the chunks of every step as
  // launch entries (forward: step 0 first; adjoint: the last step first), entry e reading
  // the outputs of entries dep_idx[dep_off[e] .. dep_off[e + 1]) (also as rows: deps,
  // LevelArgs::deps); a flag per entry and right-hand side.  Boundary b of the sweep lives in fbuf[b] (fbuf[0] = buf[0],
  // fbuf[steps] = buf[1], the others of their own).
  struct Flow {
    std::vector<int32_t> dep_off, dep_idx, deps, first_use;
    std::vector<std::pair<int32_t, int32_t>> nodes;  // per entry: (step of the launch, chunk)
    bfly::BatchEntry *entries = nullptr;
    int32_t *deps_d = nullptr, *dep_off_d = nullptr, *dep_idx_d = nullptr, *first_use_d = nullptr;
    unsigned *flags = nullptr;
    int n_entries = 0;
  };
  bool dataflow = false;
  Flow flowF, flowA;
  std::vector<void *> fbuf;
  unsigned *epoch = nullptr;                  // [2]: forward, adjoint (launches completed)
  unsigned long long *flow_sched = nullptr;  // [2][2] work counters of the two launches
  bfly_plan_info_t info{};
};

namespace bfly_state {

// Records `msg` as the calling thread's last error and returns `s`.
bfly_status set_error(bfly_status s, const std::string &msg);

inline bfly::PointArgs point_args(bfly_plan_t P, bool x_side, const void *vin, void *vout, int nrhs,
                           bool io64, bool conj, int64_t tile_rhs) {
  bfly::PointArgs a{};
  a.vin = vin;
  a.vout = vout;
  a.nrhs = nrhs;
  a.io64 = io64;
  a.conj = conj;
  a.tile_rhs = tile_rhs;
  a.tile_stride = P->TS;
  const bfly::HostTree &T = x_side ? P->TX : P->TK;
  a.n_total = T.n;
  a.nbox = T.nbox(P->L);
  a.perm = x_side ? P->perm_x : P->perm_k;
  a.leaf_start = x_side ? P->leaf_x : P->leaf_k;
  a.point_leaf = x_side ? P->pleaf_x : P->pleaf_k;
  a.W = x_side ? P->Wx : P->Wk;
  return a;
}

// Arguments of step s (forward: from boundary s to s + 1; adjoint: the reverse).
inline bfly::LevelArgs level_args(bfly_plan_t P, int s, bool adjoint, int nrhs) {
  bfly::LevelArgs a{};
  const bfly_plan_s::Step &st = P->steps[s];
  const int t_hi = st.t + 1, t_lo = st.t - st.levels + 1;  // stages of the boundaries
  void *b0 = P->buf[s & 1], *b1 = P->buf[(s + 1) & 1];
  const bfly::StageProgram &pg = adjoint ? P->progA[s] : P->progF[s];
  const bfly_plan_s::DevProg &dp = adjoint ? P->dA[s] : P->dF[s];
  a.in = adjoint ? b1 : b0;
  a.out = adjoint ? b0 : b1;
  a.in_rhs = (adjoint ? P->pairs[t_lo] : P->pairs[t_hi]) * P->TS;
  a.out_rhs = (adjoint ? P->pairs[t_hi] : P->pairs[t_lo]) * P->TS;
  a.nrhs = nrhs;
  a.chunks = dp.chunks;
  a.nchunks = (int)pg.chunks.size();
  a.blob = dp.blob;
  a.runs = dp.runs;
  a.cap0 = P->caps.cap0;
  a.cap1 = P->caps.cap1;
  a.meta_bytes = P->caps.meta_bytes;
  const bool stall = (P->flags & BFLY_FLAG_TEST_STALL) != 0;
  a.wait_limit = stall ? 2000000LL : 2000000000LL;  // ~1 ms / ~1 s of SM clock
  a.status = P->status;
  a.inject_stall = stall ? 1 : 0;
  a.sched = P->sched + ((adjoint ? P->steps.size() : 0) + (size_t)s) * 2;
  return a;
}

// Arguments of the single-launch sweep (BFLY_FLAG_DATAFLOW) in one direction.
inline bfly::LevelArgs flow_args(bfly_plan_t P, bool adjoint, int nrhs) {
  const bfly_plan_s::Flow &F = adjoint ? P->flowA : P->flowF;
  bfly::LevelArgs a = level_args(P, 0, adjoint, nrhs);
  a.in = a.out = nullptr;
  a.chunks = nullptr;
  a.blob = nullptr;
  a.runs = nullptr;
  a.entries = F.entries;
  a.nchunks = F.n_entries;
  a.sched = P->flow_sched + (adjoint ? 2 : 0);
  a.deps = F.deps_d;
  a.dep_off = F.dep_off_d;
  a.dep_idx = F.dep_idx_d;
  a.first_use = F.first_use_d;
  a.flags = F.flags;
  a.epoch = P->epoch + (adjoint ? 1 : 0);
  return a;
}


}  // namespace bfly_state
