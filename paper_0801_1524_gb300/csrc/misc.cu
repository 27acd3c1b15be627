// Launchers of the plan-time weight kernel and of the direct-sum kernel.
#include "direct.cuh"
#include "kernels.hpp"
#include "points.cuh"

namespace bfly {

cudaError_t launch_weights(int prec, int64_t n, int dim, int p, int kind, const double *off,
                           const double *inv_den, void *W, cudaStream_t s) {
  const int64_t work = n * dim;
  if (work == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((work + 255) / 256);
  if (prec == 0)
    weights_kernel<double><<<blocks, 256, 0, s>>>(n, dim, p, kind, off, inv_den, reinterpret_cast<double2 *>(W));
  else
    weights_kernel<float><<<blocks, 256, 0, s>>>(n, dim, p, kind, off, inv_den, reinterpret_cast<float2 *>(W));
  return cudaGetLastError();
}

cudaError_t launch_direct(int prec, int dim, double N, int64_t nt, const double *xt, int64_t ns,
                          const double *xs, const void *in, void *out, int nrhs, bool io64,
                          double sign, cudaStream_t s) {
  if (nt == 0 || nrhs == 0) return cudaSuccess;
  dim3 grid((unsigned)((nt + kDirectTile - 1) / kDirectTile), (unsigned)nrhs);
  if (prec == 0)
    direct_kernel<double><<<grid, kDirectTile, 0, s>>>(dim, 1.0 / N, nt, xt, ns, xs, in, out, io64, sign);
  else
    direct_kernel<float><<<grid, kDirectTile, 0, s>>>(dim, 1.0 / N, nt, xt, ns, xs, in, out, io64, sign);
  return cudaGetLastError();
}

}  // namespace bfly
