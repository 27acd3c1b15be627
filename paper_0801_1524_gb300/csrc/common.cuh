// Device helpers shared by the butterfly kernels: complex arithmetic on float2/double2
// and the argument blocks of every kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "plan.hpp"

namespace bfly {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

__device__ __forceinline__ float2 cmk(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ double2 cmk(double r, double i) { return make_double2(r, i); }

// acc + a * b
template <typename C>
__device__ __forceinline__ C cfma(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc + conj(a) * b
template <typename C>
__device__ __forceinline__ C cfma_conj(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C>
__device__ __forceinline__ C cconj(C a) {
  a.y = -a.y;
  return a;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
// FP32: one paired addition (add.rn.f32x2), rounded like the two scalar ones
template <>
__device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  return __fadd2_rn(a, b);
}
// The value of lane (lane ^ mask) of the warp (all lanes take part).
template <typename C>
__device__ __forceinline__ C shfl_xor_c(C a, int mask) {
  a.x = __shfl_xor_sync(0xffffffffu, a.x, mask);
  a.y = __shfl_xor_sync(0xffffffffu, a.y, mask);
  return a;
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with the
// programmatic stream-serialisation attribute (launch_dependent below) may be scheduled
// while its predecessor in the stream is still draining.  pdl_wait() returns once the
// predecessor grid has completed and its memory operations are visible; every thread
// calls it before its first access to memory that an earlier kernel writes or reads.
// pdl_trigger() lets the successor be scheduled before this grid ends.  Both are no-ops
// in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Launches kernel k with the programmatic stream-serialisation attribute set.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<Args &&>(args)...);
}

// Loads element i of an interleaved complex array of float or double as C.
template <typename C>
__device__ __forceinline__ C load_io(const void *p, int64_t i, bool io64) {
  if (io64) {
    const double2 v = reinterpret_cast<const double2 *>(p)[i];
    C r;
    r.x = v.x;
    r.y = v.y;
    return r;
  }
  const float2 v = reinterpret_cast<const float2 *>(p)[i];
  C r;
  r.x = v.x;
  r.y = v.y;
  return r;
}
template <typename C>
__device__ __forceinline__ void store_io(void *p, int64_t i, C v, bool io64) {
  if (io64) {
    reinterpret_cast<double2 *>(p)[i] = make_double2((double)v.x, (double)v.y);
  } else {
    reinterpret_cast<float2 *>(p)[i] = make_float2((float)v.x, (float)v.y);
  }
}

// ---------------------------------------------------------------------------------------
// Recursive step (Sec. 2.2 step 3) at one stage t, as a compiled chunk program (plan.hpp).
//   forward : in = stage t+1 charges, out = stage t charges;
//   adjoint : in = stage t, out = stage t+1.
// A stage buffer holds [rhs][tile][TS] complex values, TS = tile stride (level.cuh).
constexpr int kFlowDepRow = 64;  // ints per entry in LevelArgs::deps

struct LevelArgs {
  const void *in;
  void *out;
  int64_t in_rhs, out_rhs;      // elements between right-hand sides
  int nrhs;
  const ChunkDesc *chunks;
  int nchunks;
  const unsigned char *blob;    // per-chunk metadata blobs (plan.hpp)
  const Run *runs;
  int cap0, cap1, meta_bytes;   // shared-memory capacities the program was compiled for
  long long wait_limit;         // clock cycles before a wait gives up
  int *status;                  // device status word: bits set on a timeout
  int inject_stall;             // test hook: withhold the copies of the first chunk
  const BatchEntry *entries;    // batched launch: per-chunk chunk and buffers (else null)
  // work counter of the launch {items taken after the first round, blocks done}: zero at
  // launch, reset by the last block to finish (one per stage and direction)
  unsigned long long *sched;
  // Dataflow launch (all steps of a sweep in one launch; null otherwise).  Entries are the
  // chunks of every step, step after step; entry e reads the outputs of the entries
  // dep_idx[dep_off[e] .. dep_off[e + 1]) of the step before it, also held in the row
  // deps[e * kFlowDepRow ..] = {count, the first kFlowDepRow - 1 of them, -1 ...}.
  // flags[e * nrhs + r] holds the epoch of the last launch that published the outputs of
  // item (e, r); the launch's epoch is *epoch + 1, and the last block to finish increments
  // *epoch.
  const int *deps, *dep_off, *dep_idx;
  const int *first_use;  // per entry: the first entry that reads its outputs, -1 if none
  unsigned *flags;
  unsigned *epoch;
};

// Steps 2 and 4 and their adjoints: per-point weights against one tile per leaf.
//   spread : tile[b][l] = sum_{points j of leaf b} val_j prod_d W_j[d][l_d]
//   interp : val_i      = sum_l prod_d W_i[d][l_d] tile[leaf(i)][l]
// W is conjugated for the adjoint kinds.  val is the caller's array (I/O dtype), indexed
// through perm; tiles are the stage buffer of the plan's precision.
struct PointArgs {
  const void *vin;            // spread: caller values [nrhs][n_total] ; interp: tiles
  void *vout;                 // spread: tiles ; interp: caller values
  int64_t n_total;            // points in caller order (stride between rhs of caller data)
  int64_t nbox;               // leaves
  int64_t tile_rhs;           // elements between rhs of the tile buffer
  int tile_stride;            // elements between consecutive tiles
  int nrhs;
  bool io64;                  // caller data is complex128
  bool conj;                  // use conj(W)
  const int32_t *perm;        // sorted -> caller index
  const int32_t *leaf_start;  // [nbox+1]
  const int32_t *point_leaf;  // [n] sorted point -> leaf
  const void *W;              // [n][D][P] weights (plan precision), sorted order
};

}  // namespace bfly
