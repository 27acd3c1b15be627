// Instantiates the kernel set for one p (BFLY_P) in its own translation unit, so that
// the per-p files compile in parallel.
#include "kernels.hpp"
#include "level.cuh"
#include "points.cuh"

namespace bfly {
namespace {

template <typename R, int D, int P>
struct Impl {
  using S = LevelShape<R, D, P>;
  static cudaError_t level(const LevelArgs &a, bool adjoint, int grid, size_t smem, cudaStream_t s) {
    (void)adjoint;  // the adjoint differs only in its program and operator table
    if (a.nchunks <= 0) return cudaSuccess;
    level_kernel<R, D, P><<<grid, kLevelThreads, smem, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t level_setup(size_t smem, int *blocks) {
    // The limit is a property of the kernel function, shared by every plan on the device:
    // raise it to the device's opt-in maximum (never lower it to one plan's size, which
    // would make launches of a plan with larger blocks fail).
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(level_kernel<R, D, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, level_kernel<R, D, P>, kLevelThreads, smem);
  }
  static size_t level_smem(const ChunkCaps &c) { return S::bytes(c); }
  static int meta_bytes(int cap0, int cap1, int max_out) { return S::meta_bytes(cap0, cap1, max_out); }
  static cudaError_t spread(const PointArgs &a, cudaStream_t s) {
    constexpr int PD = ipow(P, D);
    const int64_t work = a.nbox * PD;
    if (work == 0) return cudaSuccess;
    dim3 grid((unsigned)((work + kPointThreads - 1) / kPointThreads), (unsigned)a.nrhs);
    spread_kernel<R, D, P><<<grid, kPointThreads, 0, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t interp(const PointArgs &a, cudaStream_t s) {
    if (a.n_total == 0) return cudaSuccess;
    const int64_t lanes = a.n_total * kInterpLanes;
    dim3 grid((unsigned)((lanes + kPointThreads - 1) / kPointThreads), (unsigned)a.nrhs);
    interp_kernel<R, D, P><<<grid, kPointThreads, 0, s>>>(a);
    return cudaGetLastError();
  }
  static const KernelSet *get() {
    static const KernelSet ks = {&level,         &level_setup,  &level_smem, &meta_bytes,
                                 S::table_bytes, S::tile_bytes, S::TS,      &spread,
                                 &interp};
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
