// bfly_execute_noalloc: the forward transform of an existing plan with its two charge
// buffers (the sweep's scratch memory) taken from a fixed, statically allocated device
// array instead of the plan's workspace, so that the call allocates nothing.
//
// For callers that cannot allocate device memory when they run the transform: code whose
// device memory belongs to an external allocator or a fixed memory budget, code that must
// not call cudaMalloc on its execution path (it may synchronise the device, and its
// latency is unbounded), and code that runs many plans and wants them to share one fixed
// workspace instead of one workspace per plan.
//
// The array below is a file-scope __device__ variable: every GPU that loads the library
// holds it until the process exits.  In host code its name is only a stand-in for the
// symbol, not a device address; the address is obtained with cudaGetSymbolAddress on the
// first call on each device (with that device current) and cached.  Every call shares
// the array: two calls that overlap on the GPU (two streams, or two host threads) race
// on it.  Nothing in it needs clearing: every charge tile the sweep reads was written
// earlier in the same call.
#include <cstdint>
#include <mutex>
#include <string>

#include "plan_state.hpp"

namespace {

constexpr size_t kStaticWorkspaceBytes = size_t(64) << 20;  // two charge buffers of 32 MiB
constexpr size_t kStaticBufferBytes = kStaticWorkspaceBytes / 2;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];

std::mutex g_mutex;
void *g_workspace_addr[kMaxDevices] = {};

// Device address of the static workspace on the current device (first call: looked up).
bfly_status workspace_address(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices)
    return bfly_state::set_error(BFLY_ERR_UNSUPPORTED, "device ordinal beyond the static workspace table");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_workspace_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_workspace);
    if (e != cudaSuccess || !p)
      return bfly_state::set_error(BFLY_ERR_CUDA, std::string("cudaGetSymbolAddress of the static workspace: ") +
                                                      cudaGetErrorString(e));
    g_workspace_addr[dev] = p;
  }
  *out = g_workspace_addr[dev];
  return BFLY_OK;
}

#define NOALLOC_CUDA(call)                                                                  \
  do {                                                                                      \
    const cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                                  \
      return bfly_state::set_error(BFLY_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" bfly_status bfly_execute_noalloc(bfly_plan_t plan, const void *f, void *u, int nrhs,
                                            int dtype, void *stream) {
  using bfly_state::level_args;
  using bfly_state::point_args;
  bfly_state::set_error(BFLY_OK, "");
  if (!plan) return bfly_state::set_error(BFLY_ERR_INVALID_ARG, "plan is NULL");
  if (!plan->dmem) return bfly_state::set_error(BFLY_ERR_INVALID_ARG, "plan was created host-only");
  if ((!f && plan->nk > 0) || (!u && plan->nx > 0))
    return bfly_state::set_error(BFLY_ERR_INVALID_ARG, "data pointer is NULL");
  if (nrhs < 1 || nrhs > plan->max_nrhs)
    return bfly_state::set_error(BFLY_ERR_INVALID_ARG, "nrhs outside 1..max_nrhs");
  if (dtype != BFLY_C64 && dtype != BFLY_C128) return bfly_state::set_error(BFLY_ERR_INVALID_ARG, "unknown dtype");
  int64_t max_pairs = 0;
  for (int64_t v : plan->pairs) max_pairs = v > max_pairs ? v : max_pairs;
  const size_t need = (size_t)max_pairs * plan->TS * plan->elem_bytes * (size_t)nrhs;
  if (need > kStaticBufferBytes)
    return bfly_state::set_error(
        BFLY_ERR_INVALID_ARG, "charge buffer of " + std::to_string(need) + " bytes exceeds the static workspace (" +
                                  std::to_string(kStaticBufferBytes) + " bytes per buffer, 64 MiB in all)");
  int dev = -1;
  NOALLOC_CUDA(cudaGetDevice(&dev));
  if (dev != plan->device) return bfly_state::set_error(BFLY_ERR_INVALID_ARG, "the plan belongs to another device");
  void *base = nullptr;
  const bfly_status st = workspace_address(dev, &base);
  if (st != BFLY_OK) return st;
  void *buf[2] = {base, static_cast<unsigned char *>(base) + kStaticBufferBytes};

  // the forward sweep of bfly_execute, on the static buffers
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool io64 = dtype == BFLY_C128;
  if (plan->nx == 0) return BFLY_OK;  // no targets
  if (plan->nk == 0) {                // no sources: every potential is zero
    NOALLOC_CUDA(cudaMemsetAsync(u, 0, (size_t)nrhs * plan->nx * (io64 ? 16 : 8), s));
    return BFLY_OK;
  }
  const int L = plan->L, TS = plan->TS, S = (int)plan->steps.size();
  // boundary b of the sweep (b = 0: stage L, b = S: stage 0) in buf[b mod 2]
  NOALLOC_CUDA(plan->ks->spread(point_args(plan, false, f, buf[0], nrhs, io64, false,
                                           plan->pairs[L] * TS), s));
  for (int si = 0; si < S; ++si) {
    bfly::LevelArgs a = level_args(plan, si, false, nrhs);
    a.in = buf[si & 1];
    a.out = buf[(si + 1) & 1];
    NOALLOC_CUDA(plan->ks->level(a, false, plan->level_grid, plan->level_smem, s));
  }
  NOALLOC_CUDA(plan->ks->interp(point_args(plan, true, buf[S & 1], u, nrhs, io64, false, plan->pairs[0] * TS), s));
  return BFLY_OK;
}
