// Instantiates the kernel set for one p (BFLY_P) in its own translation unit, so that
// the per-p files compile in parallel.
#include "kernels.hpp"
#include "level.cuh"
#include "points.cuh"

namespace bfly {
namespace {

template <typename R, int D, int P>
struct Impl {
  using S = LevelSmem<R, D, P>;
  static cudaError_t level(const LevelArgs &a, bool adjoint, int grid, size_t smem, cudaStream_t s) {
    if (a.nchunks <= 0) return cudaSuccess;
    if (adjoint)
      level_kernel<R, D, P, true, kLevelThreads><<<grid, kLevelThreads, smem, s>>>(a);
    else
      level_kernel<R, D, P, false, kLevelThreads><<<grid, kLevelThreads, smem, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t level_setup(size_t smem, int *blocks) {
    cudaError_t e;
    e = cudaFuncSetAttribute(level_kernel<R, D, P, false, kLevelThreads>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(level_kernel<R, D, P, true, kLevelThreads>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks, level_kernel<R, D, P, false, kLevelThreads>, kLevelThreads, smem);
  }
  static size_t level_smem(int tile_cap) { return S::bytes(tile_cap); }
  static cudaError_t spread(const PointArgs &a, cudaStream_t s) {
    constexpr int PD = ipow(P, D);
    const int64_t work = a.nbox * PD;
    if (work == 0) return cudaSuccess;
    dim3 grid((unsigned)((work + 255) / 256), (unsigned)a.nrhs);
    spread_kernel<R, D, P><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t interp(const PointArgs &a, cudaStream_t s) {
    if (a.n_total == 0) return cudaSuccess;
    dim3 grid((unsigned)((a.n_total + 255) / 256), (unsigned)a.nrhs);
    interp_kernel<R, D, P><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
  }
  static const KernelSet *get() {
    static const KernelSet ks = {&level, &level_setup, &level_smem, S::fixed_bytes, S::tile_bytes,
                                 &spread, &interp};
    return &ks;
  }
};

}  // namespace

#define BFLY_CAT2(a, b) a##b
#define BFLY_CAT(a, b) BFLY_CAT2(a, b)
const KernelSet *BFLY_CAT(kernels_p, BFLY_P)(int prec, int dim) {
  if (dim == 2) return prec == 0 ? Impl<double, 2, BFLY_P>::get() : Impl<float, 2, BFLY_P>::get();
  if (dim == 3) return prec == 0 ? Impl<double, 3, BFLY_P>::get() : Impl<float, 3, BFLY_P>::get();
  return nullptr;
}

}  // namespace bfly
