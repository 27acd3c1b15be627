// Recursive step of the butterfly (Sec. 2.2 step 3, Fig. 1), one launch per stage.
//
// For every pair (A, B) at stage t the charges are
//     f^{AB} = sum_{c in children(B)} ( (x)_d T^{(alpha_d(A), delta_d(c))} ) f^{A' Bc}
// with A' the parent of A and T the per-axis transfer operators (plan.cpp).  Work is
// grouped by unit (A', B): its inputs f^{A'Bc} are read once and shared by the outputs
// f^{AB} of every child A of A' (forward); the adjoint reads f^{AB} of the children A
// and writes f^{A'Bc} of the children Bc, with conjugate-transposed operators.
//
// A persistent block walks over chunks of consecutive units (planned on the host so
// that the chunk's tiles fit in shared memory), stages the input tiles in shared
// memory, applies the operator of axis 0..D-2 fibre by fibre into one scratch tile per
// (output, input) job, and applies the last axis while summing the jobs of an output,
// writing the result straight to global memory.
#pragma once

#include "common.cuh"

namespace bfly {

template <typename R, int D, int P>
struct LevelSmem {
  using C = typename Cx<R>::T;
  static constexpr int Q = P - 1;
  static constexpr int NOPS = 4 * Q;
  static constexpr int PD = ipow(P, D);
  static constexpr size_t table_bytes = (size_t)NOPS * P * P * sizeof(C);
  // per unit: iAp, iB, a0, c0, olo, nin, nout
  static constexpr size_t unit_bytes = (size_t)kMaxUnits * 7 * sizeof(int);
  // per input: global tile (int64) + code ; per output: global tile, code, job base,
  // input base, input count
  static constexpr size_t in_bytes = (size_t)kMaxIn * (sizeof(int64_t) + sizeof(uint32_t));
  static constexpr size_t out_bytes = (size_t)kMaxOut * (sizeof(int64_t) + 4 * sizeof(int));
  static constexpr size_t fixed_bytes = table_bytes + unit_bytes + in_bytes + out_bytes + 64 * sizeof(int);
  static constexpr size_t tile_bytes = (size_t)PD * sizeof(C);
  // per tile of capacity: the tile and one job->output map entry
  static size_t bytes(int tile_cap) {
    size_t b = fixed_bytes + (size_t)tile_cap * sizeof(uint16_t);
    b = (b + 15) & ~(size_t)15;
    return b + (size_t)tile_cap * tile_bytes;
  }
};

template <typename R, int D, int P, bool ADJ, int NT>
__global__ void __launch_bounds__(NT) level_kernel(const LevelArgs a) {
  using C = typename Cx<R>::T;
  using S = LevelSmem<R, D, P>;
  constexpr int PD = S::PD, FIB = PD / P, NOPS = S::NOPS;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *ptr = smem;
  C *s_table = reinterpret_cast<C *>(ptr);
  ptr += S::table_bytes;
  int *s_u = reinterpret_cast<int *>(ptr);  // [7][kMaxUnits]
  ptr += S::unit_bytes;
  int64_t *s_in_g = reinterpret_cast<int64_t *>(ptr);
  uint32_t *s_in_code = reinterpret_cast<uint32_t *>(s_in_g + kMaxIn);
  ptr += S::in_bytes;
  int64_t *s_out_g = reinterpret_cast<int64_t *>(ptr);
  uint32_t *s_out_code = reinterpret_cast<uint32_t *>(s_out_g + kMaxOut);
  int *s_out_jb = reinterpret_cast<int *>(s_out_code + kMaxOut);
  int *s_out_inb = s_out_jb + kMaxOut;
  int *s_out_nin = s_out_inb + kMaxOut;
  ptr += S::out_bytes;
  int *s_tmp = reinterpret_cast<int *>(ptr);  // scan scratch + totals
  ptr += 64 * sizeof(int);
  uint16_t *s_job_out = reinterpret_cast<uint16_t *>(ptr);
  ptr += (size_t)a.tile_cap * sizeof(uint16_t);
  ptr = smem + ((size_t)(ptr - smem + 15) & ~(size_t)15);
  C *s_tiles = reinterpret_cast<C *>(ptr);

  const int tid = threadIdx.x;
  const C *table = reinterpret_cast<const C *>(a.table);
  for (int e = tid; e < NOPS * P * P; e += NT) s_table[e] = table[e];

  int *u_iAp = s_u, *u_iB = s_u + kMaxUnits, *u_a0 = s_u + 2 * kMaxUnits, *u_c0 = s_u + 3 * kMaxUnits;
  int *u_olo = s_u + 4 * kMaxUnits, *u_nin = s_u + 5 * kMaxUnits, *u_nout = s_u + 6 * kMaxUnits;

  const C *gin = reinterpret_cast<const C *>(a.in);
  C *gout = reinterpret_cast<C *>(a.out);

  for (int ch = blockIdx.x; ch < a.nchunks; ch += gridDim.x) {
    const Chunk c = a.chunks[ch];
    // ---- 1. the chunk's units and their input/output/job counts
    int nin = 0, nout = 0, njob = 0;
    if (tid < c.nu) {
      const int64_t u = c.u0 + tid;
      const int iAp = (int)(u / a.nB), iB = (int)(u % a.nB);
      const int a0 = a.xcs[iAp], a1 = a.xcs[iAp + 1];
      const int c0 = a.kcs[iB], c1 = a.kcs[iB + 1];
      const int na = a1 - a0, nc = c1 - c0;
      nin = ADJ ? na : nc;
      const int full = ADJ ? nc : na;
      const int olo = c.nu == 1 ? (int)c.o_lo : 0;
      const int ohi = c.nu == 1 ? min((int)c.o_hi, full) : full;
      nout = ohi - olo;
      njob = nin * nout;
      u_iAp[tid] = iAp;
      u_iB[tid] = iB;
      u_a0[tid] = a0;
      u_c0[tid] = c0;
      u_olo[tid] = olo;
      u_nin[tid] = nin;
      u_nout[tid] = nout;
    }
    int tot_in, tot_out, tot_job;
    const int inb = block_exclusive_scan<NT>(nin, s_tmp, &tot_in);
    const int outb = block_exclusive_scan<NT>(nout, s_tmp, &tot_out);
    const int jobb = block_exclusive_scan<NT>(njob, s_tmp, &tot_job);
    // ---- 2. input / output records and the job -> output map
    if (tid < c.nu) {
      const int iAp = u_iAp[tid], iB = u_iB[tid], a0 = u_a0[tid], c0 = u_c0[tid], olo = u_olo[tid];
      for (int i = 0; i < nin; ++i) {
        if (ADJ) {
          s_in_g[inb + i] = (int64_t)(a0 + i) * a.in_row + iB;
          s_in_code[inb + i] = a.xcode[a0 + i];
        } else {
          s_in_g[inb + i] = (int64_t)iAp * a.in_row + (c0 + i);
          s_in_code[inb + i] = a.kcode[c0 + i];
        }
      }
      for (int o = 0; o < nout; ++o) {
        const int oo = olo + o;
        if (ADJ) {
          s_out_g[outb + o] = (int64_t)iAp * a.out_row + (c0 + oo);
          s_out_code[outb + o] = a.kcode[c0 + oo];
        } else {
          s_out_g[outb + o] = (int64_t)(a0 + oo) * a.out_row + iB;
          s_out_code[outb + o] = a.xcode[a0 + oo];
        }
        s_out_jb[outb + o] = jobb + o * nin;
        s_out_inb[outb + o] = inb;
        s_out_nin[outb + o] = nin;
        for (int i = 0; i < nin; ++i) s_job_out[jobb + o * nin + i] = (uint16_t)(outb + o);
      }
    }
    __syncthreads();
    C *s_scr = s_tiles + (size_t)tot_in * PD;

    for (int r = 0; r < a.nrhs; ++r) {
      const C *rin = gin + (size_t)r * a.in_rhs;
      C *rout = gout + (size_t)r * a.out_rhs;
      // ---- 3. stage the input tiles
      for (int e = tid; e < tot_in * PD; e += NT) {
        const int t = e / PD, l = e - t * PD;
        s_tiles[e] = rin[s_in_g[t] * PD + l];
      }
      __syncthreads();
      // ---- 4. axes 0 .. D-2, one scratch tile per job
#pragma unroll
      for (int k = 0; k < D - 1; ++k) {
        const int sk = ipow(P, D - 1 - k);  // element stride of axis k
        for (int w = tid; w < tot_job * FIB; w += NT) {
          const int j = w / FIB, f = w - j * FIB;
          const int o = s_job_out[j];
          const int i = j - s_out_jb[o];
          const int tin = s_out_inb[o] + i;
          const uint32_t ic = s_in_code[tin], oc = s_out_code[o];
          const uint32_t xc = ADJ ? ic : oc, kc = ADJ ? oc : ic;
          const int op = (int)((xc >> (8 * k)) & 0xffu) * 2 + (int)((kc >> k) & 1u);
          const C *src = (k == 0) ? (s_tiles + (size_t)tin * PD) : (s_scr + (size_t)j * PD);
          C *dst = s_scr + (size_t)j * PD;
          const int base = (f / sk) * sk * P + (f % sk);
          C x[P];
#pragma unroll
          for (int l = 0; l < P; ++l) x[l] = src[base + l * sk];
          const C *T = s_table + (size_t)op * P * P;
#pragma unroll
          for (int m = 0; m < P; ++m) {
            C y = cmk((R)0, (R)0);
#pragma unroll
            for (int l = 0; l < P; ++l) y = cfma(T[m * P + l], x[l], y);
            dst[base + m * sk] = y;
          }
        }
        __syncthreads();
      }
      // ---- 5. last axis, sum over the jobs of each output, store
      for (int w = tid; w < tot_out * FIB; w += NT) {
        const int o = w / FIB, f = w - o * FIB;
        const uint32_t oc = s_out_code[o];
        const int jb = s_out_jb[o], ib = s_out_inb[o], ni = s_out_nin[o];
        C acc[P];
#pragma unroll
        for (int m = 0; m < P; ++m) acc[m] = cmk((R)0, (R)0);
        for (int i = 0; i < ni; ++i) {
          const uint32_t ic = s_in_code[ib + i];
          const uint32_t xc = ADJ ? ic : oc, kc = ADJ ? oc : ic;
          const int op = (int)((xc >> (8 * (D - 1))) & 0xffu) * 2 + (int)((kc >> (D - 1)) & 1u);
          const C *src = s_scr + (size_t)(jb + i) * PD + f * P;
          C x[P];
#pragma unroll
          for (int l = 0; l < P; ++l) x[l] = src[l];
          const C *T = s_table + (size_t)op * P * P;
#pragma unroll
          for (int m = 0; m < P; ++m) {
#pragma unroll
            for (int l = 0; l < P; ++l) acc[m] = cfma(T[m * P + l], x[l], acc[m]);
          }
        }
        C *dst = rout + s_out_g[o] * PD + f * P;
#pragma unroll
        for (int m = 0; m < P; ++m) dst[m] = acc[m];
      }
      __syncthreads();
    }
  }
}

}  // namespace bfly
