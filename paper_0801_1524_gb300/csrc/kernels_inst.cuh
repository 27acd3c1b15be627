// Instantiates the kernel set for one p (BFLY_P) in its own translation unit, so that
// the per-p files compile in parallel.
#include <mutex>
#include <vector>

#include <cstring>

#include "kernels.hpp"
#include "level.cuh"
#include "level_tc.cuh"
#include "points.cuh"

namespace bfly {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_ops_mutex;
bool g_ops_ready[kMaxDevices][2] = {};  // [device][FP32?]

// Writes the factors of the transfer operators of this p (both directions, FP64-built,
// rounded once to the precision R) to constant memory of the current device, the first
// time only: they are the same for every plan, so later plans find them in place.
template <typename R>
cudaError_t init_operators() {
  using C = typename Cx<R>::T;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_ops_mutex);
  bool &ready = g_ops_ready[dev][sizeof(R) == 4];
  if (ready) return cudaSuccess;
  constexpr int P = BFLY_P;
  std::vector<C> w((size_t)2 * 2 * P * P), phi((size_t)2 * 2 * P);
  std::vector<float4> wp(w.size()), phip(phi.size());  // FP32: packed (re, re, -im, im)
  std::vector<double> wd((size_t)2 * P * P * 2), pd((size_t)2 * P * 2);
  auto pack = [](double re, double im) {
    return make_float4((float)re, (float)re, -(float)im, (float)im);
  };
  for (int adj = 0; adj < 2; ++adj) {
    transfer_factors(P, adj != 0, wd.data(), pd.data());
    for (int i = 0; i < 2 * P * P; ++i) {
      C c;
      c.x = (R)wd[2 * i];
      c.y = (R)wd[2 * i + 1];
      w[(size_t)adj * 2 * P * P + i] = c;
      wp[(size_t)adj * 2 * P * P + i] = pack(wd[2 * i], wd[2 * i + 1]);
    }
    for (int i = 0; i < 2 * P; ++i) {
      C c;
      c.x = (R)pd[2 * i];
      c.y = (R)pd[2 * i + 1];
      phi[(size_t)adj * 2 * P + i] = c;
      phip[(size_t)adj * 2 * P + i] = pack(pd[2 * i], pd[2 * i + 1]);
    }
  }
  if constexpr (sizeof(R) == 4) {
    e = cudaMemcpyToSymbol(c_w32, wp.data(), wp.size() * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_phi32, phip.data(), phip.size() * sizeof(float4));
  } else {
    e = cudaMemcpyToSymbol(c_w64, w.data(), w.size() * sizeof(C));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_phi64, phi.data(), phi.size() * sizeof(C));
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) ready = true;
  return e;
}

bool g_tc_ready[kMaxDevices] = {};

// v rounded to TF32 (10 explicit mantissa bits, to nearest even), as a float.
float tf32_round(double v) {
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x0fffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
  }
  std::memcpy(&f, &u, 4);
  return f;
}

// Writes the A fragments of the tensor-core recursive step (level_tc.cuh) of this p to
// the device table g_tc_frag, the first time on the current device: for both directions
// and op = gamma*2 + delta the complex operator (forward C = W(delta) diag(phi_gamma),
// adjoint C^H = diag(conj phi_gamma) W(delta)^H, from the FP64 factors), its real form
// R[2m + c'][2l + c] (re -im / im re blocks) zero-padded to 16 MT x 8 KT, and per lane
// (g, t4) of every (m16, k8) tile a0..a3 = R[g][t4], R[g+8][t4], R[g][t4+4], R[g+8][t4+4],
// split as hi = tf32(R), lo = tf32(R - hi).
cudaError_t init_tc_operators() {
  constexpr int P = BFLY_P;
  constexpr int MT = (2 * P + 15) / 16, KT = (2 * P + 7) / 8;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_ops_mutex);
  if (g_tc_ready[dev]) return cudaSuccess;
  std::vector<float4> frag((size_t)2 * 4 * MT * KT * 2 * 32);
  std::vector<double> wd((size_t)2 * P * P * 2), pd((size_t)2 * P * 2);
  std::vector<double> R((size_t)16 * MT * 8 * KT);
  for (int adj = 0; adj < 2; ++adj) {
    transfer_factors(P, adj != 0, wd.data(), pd.data());
    for (int op = 0; op < 4; ++op) {
      const int gamma = op >> 1, delta = op & 1;
      std::fill(R.begin(), R.end(), 0.0);
      for (int m = 0; m < P; ++m)
        for (int l = 0; l < P; ++l) {
          const size_t wi = ((size_t)delta * P + m) * P + l;
          double cr = wd[2 * wi], ci = wd[2 * wi + 1];
          if (gamma) {
            const int pl = adj ? m : l;  // forward: column scaling; adjoint: row scaling
            const double fr = pd[2 * (delta * P + pl)], fi = pd[2 * (delta * P + pl) + 1];
            const double tr = cr * fr - ci * fi, ti = cr * fi + ci * fr;
            cr = tr;
            ci = ti;
          }
          R[(size_t)(2 * m) * 8 * KT + 2 * l] = cr;
          R[(size_t)(2 * m) * 8 * KT + 2 * l + 1] = -ci;
          R[(size_t)(2 * m + 1) * 8 * KT + 2 * l] = ci;
          R[(size_t)(2 * m + 1) * 8 * KT + 2 * l + 1] = cr;
        }
      for (int mt = 0; mt < MT; ++mt)
        for (int kt = 0; kt < KT; ++kt)
          for (int lane = 0; lane < 32; ++lane) {
            const int g = lane >> 2, t4 = lane & 3;
            const double v[4] = {R[(size_t)(16 * mt + g) * 8 * KT + 8 * kt + t4],
                                 R[(size_t)(16 * mt + g + 8) * 8 * KT + 8 * kt + t4],
                                 R[(size_t)(16 * mt + g) * 8 * KT + 8 * kt + t4 + 4],
                                 R[(size_t)(16 * mt + g + 8) * 8 * KT + 8 * kt + t4 + 4]};
            float hi[4], lo[4];
            for (int i = 0; i < 4; ++i) {
              hi[i] = tf32_round(v[i]);
              lo[i] = tf32_round(v[i] - (double)hi[i]);
            }
            const size_t at = ((((size_t)adj * 4 + op) * MT + mt) * KT + kt) * 2 * 32;
            frag[at + lane] = make_float4(hi[0], hi[1], hi[2], hi[3]);
            frag[at + 32 + lane] = make_float4(lo[0], lo[1], lo[2], lo[3]);
          }
    }
  }
  e = cudaMemcpyToSymbol(g_tc_frag, frag.data(), frag.size() * sizeof(float4));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) g_tc_ready[dev] = true;
  return e;
}

template <typename R, int D, int P>
struct Impl {
  using S = LevelShape<R, D, P>;
  static cudaError_t level(const LevelArgs &a, bool adjoint, int grid, size_t smem, cudaStream_t s) {
    if (a.nchunks <= 0) return cudaSuccess;
    if (a.deps)
      return launch_dependent(adjoint ? level_kernel<R, D, P, true, true> : level_kernel<R, D, P, false, true>,
                              dim3(grid), dim3(kLevelThreads), smem, s, a);
    return launch_dependent(adjoint ? level_kernel<R, D, P, true, false> : level_kernel<R, D, P, false, false>,
                            dim3(grid), dim3(kLevelThreads), smem, s, a);
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
    for (auto k : {level_kernel<R, D, P, false, false>, level_kernel<R, D, P, true, false>,
                   level_kernel<R, D, P, false, true>, level_kernel<R, D, P, true, true>})
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) e = init_operators<R>();
    if (e != cudaSuccess) return e;
    int b2 = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, level_kernel<R, D, P, false, false>, kLevelThreads, smem);
    for (auto k : {level_kernel<R, D, P, true, false>, level_kernel<R, D, P, false, true>,
                   level_kernel<R, D, P, true, true>}) {
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k, kLevelThreads, smem);
      if (e == cudaSuccess && b2 < *blocks) *blocks = b2;
    }
    return e;
  }
  static size_t level_smem(const ChunkCaps &c) { return S::bytes(c); }
  static int meta_bytes(int cap0, int cap1, int max_out) { return S::meta_bytes(cap0, cap1, max_out); }
  static cudaError_t spread(const PointArgs &a, cudaStream_t s) {
    constexpr int PD = ipow(P, D);
    const int64_t work = a.nbox * PD;
    if (work == 0) return cudaSuccess;
    constexpr int64_t E = kPointThreads * kSpreadPerThread;
    dim3 grid((unsigned)((work + E - 1) / E), (unsigned)((a.nrhs + kPointRhs - 1) / kPointRhs));
    return launch_dependent(spread_kernel<R, D, P>, grid, dim3(kPointThreads), 0, s, a);
  }
  static cudaError_t interp(const PointArgs &a, cudaStream_t s) {
    if (a.n_total == 0) return cudaSuccess;
    const int64_t lanes = a.n_total * kInterpLanes;
    dim3 grid((unsigned)((lanes + kPointThreads - 1) / kPointThreads), (unsigned)((a.nrhs + kPointRhs - 1) / kPointRhs));
    return launch_dependent(interp_kernel<R, D, P>, grid, dim3(kPointThreads), 0, s, a);
  }
  static const KernelSet *get() {
    static const KernelSet ks = {&level, &level_setup, &level_smem, &meta_bytes, S::tile_bytes, S::TS, &spread,
                                 &interp};
    return &ks;
  }
};

// The FP32 kernel sets with the recursive step on groups of eight right-hand sides
// (level_tc_kernel): on the tensor cores (MMA) or with paired FP32 multiply-adds; the leaf
// and final steps and the charge layout are those of the FP32 set.
template <int D, int P, bool MMA>
struct ImplTc {
  using S = TcShape<D, P>;
  static cudaError_t level(const LevelArgs &a, bool adjoint, int grid, size_t smem, cudaStream_t s) {
    if (a.nchunks <= 0) return cudaSuccess;
    return launch_dependent(adjoint ? level_tc_kernel<D, P, true, MMA> : level_tc_kernel<D, P, false, MMA>, dim3(grid),
                            dim3(kLevelThreads), smem, s, a);
  }
  static cudaError_t level_setup(size_t smem, int *blocks) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(level_tc_kernel<D, P, false, MMA>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(level_tc_kernel<D, P, true, MMA>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) e = MMA ? init_tc_operators() : init_operators<float>();
    if (e != cudaSuccess) return e;
    int b2 = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, level_tc_kernel<D, P, false, MMA>, kLevelThreads, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, level_tc_kernel<D, P, true, MMA>, kLevelThreads, smem);
    if (b2 < *blocks) *blocks = b2;
    return e;
  }
  static size_t level_smem(const ChunkCaps &c) { return S::bytes(c); }
  static const KernelSet *get() {
    using F = Impl<float, D, P>;
    static const KernelSet ks = {&level, &level_setup, &level_smem, &F::meta_bytes, S::tile_bytes, S::TS,
                                 &F::spread, &F::interp};
    return &ks;
  }
};

}  // namespace

#define BFLY_CAT2(a, b) a##b
#define BFLY_CAT(a, b) BFLY_CAT2(a, b)
const KernelSet *BFLY_CAT(kernels_p, BFLY_P)(int prec, int dim) {
  if (prec == 2) return dim == 2 ? ImplTc<2, BFLY_P, true>::get() : nullptr;
  if (prec == 3) return dim == 2 ? ImplTc<2, BFLY_P, false>::get() : nullptr;
  if (dim == 2) return prec == 0 ? Impl<double, 2, BFLY_P>::get() : Impl<float, 2, BFLY_P>::get();
  if (dim == 3) return prec == 0 ? Impl<double, 3, BFLY_P>::get() : Impl<float, 3, BFLY_P>::get();
  return nullptr;
}

}  // namespace bfly
