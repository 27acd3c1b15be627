// Launchers of the sm_103a kernels, one set per (precision, dimension, p).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace bfly {

struct KernelSet {
  // recursive step at one stage; grid = persistent blocks, smem = dynamic bytes
  cudaError_t (*level)(const LevelArgs &a, bool adjoint, int grid, size_t smem, cudaStream_t s);
  // raises the dynamic shared memory limit to the device maximum, writes the operator
  // factors to constant memory (first call on a device) and returns the blocks per SM
  // resident with `smem` bytes each
  cudaError_t (*level_setup)(size_t smem, int *blocks_per_sm);
  size_t (*level_smem)(const ChunkCaps &caps);
  int (*meta_bytes)(int cap0, int cap1, int max_out);
  size_t level_tile_bytes;
  int tile_stride;  // complex elements per stored charge tile
  cudaError_t (*spread)(const PointArgs &a, cudaStream_t s);
  cudaError_t (*interp)(const PointArgs &a, cudaStream_t s);
};


// prec: 0 = FP64, 1 = FP32, 2 = FP32 with the recursive step on the tensor cores (2D).
// Returns nullptr when (prec, dim, p) has no kernels.
const KernelSet *kernels_p3(int prec, int dim);
const KernelSet *kernels_p5(int prec, int dim);
const KernelSet *kernels_p7(int prec, int dim);
const KernelSet *kernels_p9(int prec, int dim);

cudaError_t launch_weights(int prec, int64_t n, int dim, int p, int kind, const double *off,
                           const double *inv_den, void *W, cudaStream_t s);
cudaError_t launch_direct(int prec, int dim, double N, int64_t nt, const double *xt, int64_t ns,
                          const double *xs, const void *in, void *out, int nrhs, bool io64,
                          double sign, cudaStream_t s);

}  // namespace bfly
