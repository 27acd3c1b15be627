// The transform by its definition (eq. 1.1) on the GPU: u_i = sum_j e^{s 2 pi i x_i.k_j/N} f_j
// with s = +1 (forward) or -1 (adjoint, roles of the point sets swapped).  The phase
// x.k/N is formed in FP64 and reduced to [-1/2, 1/2] (exact), then the exponential is
// evaluated in R.  For R = float the sum over one tile of sources is FP32 and tiles are
// added in FP64; for R = double everything is FP64.
#pragma once

#include "common.cuh"

namespace bfly {

template <typename R> __device__ __forceinline__ void sincospi_r(double ph, R *s, R *c);
template <> __device__ __forceinline__ void sincospi_r<float>(double ph, float *s, float *c) {
  sincospif((float)ph, s, c);
}
template <> __device__ __forceinline__ void sincospi_r<double>(double ph, double *s, double *c) {
  sincospi(ph, s, c);
}

constexpr int kDirectTile = 256;

template <typename R>
__global__ void __launch_bounds__(kDirectTile) direct_kernel(
    int dim, double invN, int64_t nt, const double *xt, int64_t ns, const double *xs,
    const void *in, void *out, bool io64, double sign) {
  using C = typename Cx<R>::T;
  __shared__ double s_x[kDirectTile * 3];
  __shared__ C s_f[kDirectTile];
  const int64_t i = (int64_t)blockIdx.x * kDirectTile + threadIdx.x;
  const int r = blockIdx.y;
  double xi[3] = {0.0, 0.0, 0.0};
  if (i < nt)
    for (int d = 0; d < dim; ++d) xi[d] = xt[i * dim + d] * invN;
  double acc_re = 0.0, acc_im = 0.0;
  for (int64_t j0 = 0; j0 < ns; j0 += kDirectTile) {
    const int nj = (int)min((int64_t)kDirectTile, ns - j0);
    __syncthreads();
    if (threadIdx.x < nj) {
      const int64_t j = j0 + threadIdx.x;
      for (int d = 0; d < dim; ++d) s_x[threadIdx.x * 3 + d] = xs[j * dim + d];
      s_f[threadIdx.x] = load_io<C>(in, (int64_t)r * ns + j, io64);
    }
    __syncthreads();
    R tre = 0, tim = 0;
    for (int jj = 0; jj < nj; ++jj) {
      double ph = xi[0] * s_x[jj * 3];
      for (int d = 1; d < dim; ++d) ph = fma(xi[d], s_x[jj * 3 + d], ph);
      ph -= rint(ph);
      R sn, cs;
      sincospi_r<R>(2.0 * ph, &sn, &cs);
      sn *= (R)sign;
      const C f = s_f[jj];
      tre = fma(cs, f.x, tre);
      tre = fma(-sn, f.y, tre);
      tim = fma(cs, f.y, tim);
      tim = fma(sn, f.x, tim);
    }
    acc_re += (double)tre;
    acc_im += (double)tim;
  }
  if (i < nt) store_io(out, (int64_t)r * nt + i, make_double2(acc_re, acc_im), io64);
}

}  // namespace bfly
