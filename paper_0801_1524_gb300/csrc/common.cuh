// Device helpers shared by the butterfly kernels: complex arithmetic on float2/double2,
// a block-wide exclusive scan, and the argument blocks of every kernel.
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

// Exclusive scan of one int per thread over a block of NT threads (NT a multiple of 32,
// at most 1024).  `tmp` holds NT/32 ints of shared memory.  Returns the exclusive
// prefix; *total receives the block sum.  Contains __syncthreads().
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int *tmp, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < NT / 32 ? tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NT / 32) tmp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const int base = warp > 0 ? tmp[warp - 1] : 0;
  *total = tmp[NT / 32 - 1];
  __syncthreads();
  return base + incl - v;
}

// ---------------------------------------------------------------------------------------
// Recursive step (Sec. 2.2 step 3) at one stage t.
//   forward : in = stage t+1 charges [rhs][nAp][in_row][P^D], out = stage t charges
//             [rhs][nA][out_row][P^D]; unit (A', B) reads f^{A'Bc} for the children Bc
//             of B and writes f^{AB} for the children A of A'.
//   adjoint : in = stage t, out = stage t+1; the unit reads the tiles of the children A
//             of A' and writes the tiles of the children Bc of B.
struct LevelArgs {
  const void *in;
  void *out;
  int64_t in_row, out_row;    // tiles per row (number of B boxes) of in and out
  int64_t in_rhs, out_rhs;    // elements between right-hand sides
  int nrhs;
  int64_t nB;                 // B boxes at level t (units = nAp * nB)
  const int32_t *xcs;         // [nAp+1] children of A' (T_X level L-t-1 -> L-t)
  const uint32_t *xcode;      // [nA] alpha_d = a_d mod 2q, 8 bits per axis
  const int32_t *kcs;         // [nB+1] children of B (T_K level t -> t+1)
  const uint32_t *kcode;      // [nBc] delta_d = b_d & 1, 1 bit per axis
  const Chunk *chunks;
  int nchunks;
  const void *table;          // [4q][P][P] complex operators (conjugate-transposed: adjoint)
  int tile_cap;               // charge tiles of shared memory per block
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
  int nrhs;
  bool io64;                  // caller data is complex128
  bool conj;                  // use conj(W)
  const int32_t *perm;        // sorted -> caller index
  const int32_t *leaf_start;  // [nbox+1]
  const int32_t *point_leaf;  // [n] sorted point -> leaf
  const void *W;              // [n][D][P] weights (plan precision), sorted order
};

}  // namespace bfly
