// Batched execution of many plans (independent transforms of uneven N and point counts,
// each with nrhs right-hand sides; the plans share dim, p, precision and tile capacities,
// and so the operators): the leaf step of every plan, then one launch of the
// recursive-step kernel per stage t = L_max-1 .. 0 over the chunks of every plan's step
// that starts at stage t (one or two stages; plans are aligned at the final stage), then
// the final step of every
// plan.  On a non-default stream the whole sequence is captured once into a CUDA graph
// and replayed while the buffers and nrhs stay the same.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "plan_state.hpp"

struct bfly_batch_s {
  int count = 0, dim = 0, p = 0, prec = 0, L_max = 0, max_nrhs = 0, device = -1;
  int meta_bytes = 0, grid = 0;  // the largest metadata slot of the plans; persistent blocks
  size_t smem = 0;
  std::vector<bfly_plan_t> plans;
  char *dmem = nullptr;
  std::vector<bfly::BatchEntry *> entries;  // per stage t
  std::vector<int> n_entries;
  int *status = nullptr;
  unsigned long long *sched = nullptr;  // work counters of the stage launches, [t][2]
  // graph of the last execute: replayed when the key matches
  cudaGraphExec_t exec = nullptr;
  std::vector<const void *> key_f;
  std::vector<void *> key_u;
  int key_nrhs = 0, key_dtype = -1;
  cudaStream_t key_stream = nullptr;
};

namespace {

using bfly_state::point_args;
using bfly_state::set_error;

#define BATCH_CUDA(call)                                                                     \
  do {                                                                                       \
    const cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                                   \
      return set_error(e_ == cudaErrorMemoryAllocation ? BFLY_ERR_OUT_OF_MEMORY : BFLY_ERR_CUDA, \
                       std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

bfly_status launch_all(bfly_batch_t B, const void *const *f, void *const *u, int nrhs, int dtype,
                       cudaStream_t s) {
  const bool io64 = dtype == BFLY_C128;
  auto empty = [](bfly_plan_t P) { return P->nx == 0 || P->nk == 0; };
  for (int i = 0; i < B->count; ++i) {
    bfly_plan_t P = B->plans[i];
    if (empty(P)) {  // no targets: nothing; no sources: zero potentials
      if (P->nx > 0) BATCH_CUDA(cudaMemsetAsync(u[i], 0, (size_t)nrhs * P->nx * (io64 ? 16 : 8), s));
      continue;
    }
    BATCH_CUDA(P->ks->spread(point_args(P, false, f[i], P->buf[0], nrhs, io64, false,
                                        P->pairs[P->L] * P->TS), s));
  }
  bfly_plan_t P0 = B->plans[0];
  // launch t: the steps of every plan that start at stage t (one or two stages each)
  for (int t = B->L_max - 1; t >= 0; --t) {
    if (B->n_entries[t] == 0) continue;
    // the operators and tile capacities of plan 0 serve all (same dim, p, precision)
    bfly::LevelArgs a{};
    a.nrhs = nrhs;
    a.entries = B->entries[t];
    a.nchunks = B->n_entries[t];
    a.cap0 = P0->caps.cap0;
    a.cap1 = P0->caps.cap1;
    a.meta_bytes = B->meta_bytes;
    a.wait_limit = 2000000000LL;  // ~1 s of SM clock
    a.status = B->status;
    a.sched = B->sched + (size_t)t * 2;
    BATCH_CUDA(P0->ks->level(a, false, B->grid, B->smem, s));
  }
  for (int i = 0; i < B->count; ++i) {
    bfly_plan_t P = B->plans[i];
    if (empty(P)) continue;
    BATCH_CUDA(P->ks->interp(point_args(P, true, P->buf[P->steps.size() & 1], u[i], nrhs, io64, false,
                                        P->pairs[0] * P->TS), s));
  }
  return BFLY_OK;
}

}  // namespace

extern "C" {

void bfly_batch_destroy(bfly_batch_t B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->dmem) cudaFree(B->dmem);
  delete B;
}

bfly_status bfly_batch_create(bfly_batch_t *out, int count, const bfly_plan_t *plans) {
  set_error(BFLY_OK, "");
  if (!out) return set_error(BFLY_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !plans) return set_error(BFLY_ERR_INVALID_ARG, "count must be >= 1 and plans non-NULL");
  bfly_plan_t P0 = plans[0];
  for (int i = 0; i < count; ++i) {
    bfly_plan_t P = plans[i];
    if (!P || !P->dmem) return set_error(BFLY_ERR_INVALID_ARG, "every plan must be a device plan");
    if (P->dim != P0->dim || P->p != P0->p || P->prec != P0->prec || P->device != P0->device || P->ks != P0->ks)
      return set_error(BFLY_ERR_INVALID_ARG,
                       "plans of a batch share dim, p, precision, device and recursive-step kernel");
    if (P->caps.cap0 != P0->caps.cap0 || P->caps.cap1 != P0->caps.cap1 || P->caps.max_out != P0->caps.max_out)
      return set_error(BFLY_ERR_INVALID_ARG, "plans of a batch share their shared-memory tile capacities");
  }
  // one launch serves every plan: metadata slots as large as the largest plan's
  int meta = 0;
  for (int i = 0; i < count; ++i) meta = std::max(meta, plans[i]->caps.meta_bytes);
  bfly::ChunkCaps caps = P0->caps;
  caps.meta_bytes = meta;
  const size_t smem = P0->ks->level_smem(caps);
  int blocks = 0, sms = 0;
  cudaError_t es = P0->ks->level_setup(smem, &blocks);
  if (es == cudaSuccess) es = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P0->device);
  if (es != cudaSuccess) return set_error(BFLY_ERR_CUDA, std::string("batch setup: ") + cudaGetErrorString(es));
  if (blocks < 1) return set_error(BFLY_ERR_UNSUPPORTED, "the batch's blocks do not fit in shared memory");
  bfly_batch_t B = new bfly_batch_s();
  B->count = count;
  B->dim = P0->dim;
  B->p = P0->p;
  B->prec = P0->prec;
  B->device = P0->device;
  B->plans.assign(plans, plans + count);
  B->max_nrhs = P0->max_nrhs;
  B->meta_bytes = meta;
  B->smem = smem;
  B->grid = blocks * sms;
  for (auto *P : B->plans) {
    B->L_max = std::max(B->L_max, P->L);
    B->max_nrhs = std::min(B->max_nrhs, P->max_nrhs);
  }
  // entries of every stage, all plans
  std::vector<std::vector<bfly::BatchEntry>> host(B->L_max);
  for (int t = 0; t < B->L_max; ++t) {
    std::vector<double> work;  // the chunks of every plan, scheduled together
    for (auto *P : B->plans) {
      int si = 0;
      while (si < (int)P->steps.size() && P->steps[si].t != t) ++si;
      if (si == (int)P->steps.size()) continue;  // no step of this plan starts at stage t
      const int t_lo = t - P->steps[si].levels + 1;
      const bfly::StageProgram &pg = P->progF[si];
      for (const bfly::ChunkDesc &cd : pg.chunks) {
        work.push_back(bfly::chunk_work(pg.blob.data() + cd.blob_off, B->dim, B->p));
        bfly::BatchEntry e;
        e.d = cd;
        e.blob = P->dF[si].blob;
        e.runs = P->dF[si].runs;
        e.in = P->buf[si & 1];
        e.out = P->buf[(si + 1) & 1];
        e.in_rhs = P->pairs[t + 1] * P->TS;
        e.out_rhs = P->pairs[t_lo] * P->TS;
        host[t].push_back(e);
      }
    }
    const std::vector<size_t> order = bfly::schedule_chunks(work);
    std::vector<bfly::BatchEntry> sorted(host[t].size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = host[t][order[i]];
    host[t].swap(sorted);
  }
  const size_t sched_bytes = ((size_t)B->L_max * 2 * sizeof(unsigned long long) + 255) & ~(size_t)255;
  size_t total = 256 + sched_bytes;  // status word, work counters
  for (auto &v : host) total += (v.size() * sizeof(bfly::BatchEntry) + 255) & ~(size_t)255;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&B->dmem), total);
  if (e != cudaSuccess) {
    delete B;
    return set_error(BFLY_ERR_OUT_OF_MEMORY, std::string("cudaMalloc of the batch: ") + cudaGetErrorString(e));
  }
  size_t at = 0;
  B->status = reinterpret_cast<int *>(B->dmem);
  e = cudaMemset(B->status, 0, sizeof(int));
  at += 256;
  B->sched = reinterpret_cast<unsigned long long *>(B->dmem + at);
  if (e == cudaSuccess) e = cudaMemset(B->sched, 0, sched_bytes);
  at += sched_bytes;
  B->entries.assign(B->L_max, nullptr);
  B->n_entries.assign(B->L_max, 0);
  for (int t = 0; t < B->L_max && e == cudaSuccess; ++t) {
    B->entries[t] = reinterpret_cast<bfly::BatchEntry *>(B->dmem + at);
    B->n_entries[t] = (int)host[t].size();
    if (!host[t].empty())
      e = cudaMemcpy(B->entries[t], host[t].data(), host[t].size() * sizeof(bfly::BatchEntry),
                     cudaMemcpyHostToDevice);
    at += (host[t].size() * sizeof(bfly::BatchEntry) + 255) & ~(size_t)255;
  }
  if (e != cudaSuccess) {
    bfly_batch_destroy(B);
    return set_error(BFLY_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
  }
  *out = B;
  return BFLY_OK;
}

bfly_status bfly_batch_execute(bfly_batch_t B, const void *const *f, void *const *u, int nrhs, int dtype,
                               void *stream) {
  set_error(BFLY_OK, "");
  if (!B || !f || !u) return set_error(BFLY_ERR_INVALID_ARG, "batch, f or u is NULL");
  if (nrhs < 1 || nrhs > B->max_nrhs) return set_error(BFLY_ERR_INVALID_ARG, "nrhs outside 1..max_nrhs of the plans");
  if (dtype != BFLY_C64 && dtype != BFLY_C128) return set_error(BFLY_ERR_INVALID_ARG, "unknown dtype");
  for (int i = 0; i < B->count; ++i)
    if ((!f[i] && B->plans[i]->nk > 0) || (!u[i] && B->plans[i]->nx > 0))
      return set_error(BFLY_ERR_INVALID_ARG, "a data pointer is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!s) return launch_all(B, f, u, nrhs, dtype, s);  // the legacy stream cannot be captured
  const bool same = B->exec && B->key_nrhs == nrhs && B->key_dtype == dtype && B->key_stream == s &&
                    std::memcmp(B->key_f.data(), f, B->count * sizeof(void *)) == 0 &&
                    std::memcmp(B->key_u.data(), u, B->count * sizeof(void *)) == 0;
  if (!same) {
    if (B->exec) {
      cudaGraphExecDestroy(B->exec);
      B->exec = nullptr;
    }
    BATCH_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const bfly_status st = launch_all(B, f, u, nrhs, dtype, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (st != BFLY_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (ec != cudaSuccess) return set_error(BFLY_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    const cudaError_t ei = cudaGraphInstantiate(&B->exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      B->exec = nullptr;
      return set_error(BFLY_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    }
    B->key_f.assign(f, f + B->count);
    B->key_u.assign(u, u + B->count);
    B->key_nrhs = nrhs;
    B->key_dtype = dtype;
    B->key_stream = s;
  }
  BATCH_CUDA(cudaGraphLaunch(B->exec, s));
  return BFLY_OK;
}

bfly_status bfly_batch_status(bfly_batch_t B, int *flags) {
  set_error(BFLY_OK, "");
  if (!B) return set_error(BFLY_ERR_INVALID_ARG, "batch is NULL");
  int v = 0;
  BATCH_CUDA(cudaDeviceSynchronize());
  BATCH_CUDA(cudaMemcpy(&v, B->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) BATCH_CUDA(cudaMemset(B->status, 0, sizeof(int)));
  if (flags) *flags = v;
  if (v) return set_error(BFLY_ERR_TIMEOUT, "a bounded device-side wait gave up (status bits " + std::to_string(v) + ")");
  return BFLY_OK;
}

}  // extern "C"
