// Recursive step of the butterfly (Sec. 2.2 step 3) on the tensor cores, for many
// right-hand sides: the same chunk programs as level_kernel (level.cuh), with a work item
// of eight right-hand sides of a chunk instead of one.
//
// Every right-hand side of a box pair goes through the same operators, so for one item of
// a pass (an output tile, one or two source tiles, operators C^{op}) and one fibre of the
// tile along the pass's axis, the eight right-hand sides form the columns of a real
// matrix product
//     Y (2P x 8) = sum over the item's sources of  R(C^{op}) (2P x 2P) . X (2P x 8),
// R(C) the real form of the complex operator (rows and columns interleaved re, im).  It is
// issued as mma.sync m16n8k8 with TF32 operands and FP32 accumulation, compensated by
// splitting both operands, a = a_hi + a_lo with a_hi = tf32(a) and a_lo = tf32(a - a_hi):
// R X ~= R_lo X_hi + R_hi X_lo + R_hi X_hi  (three products; the dropped R_lo X_lo is
// 2^-22 relative), with the main product's sums rounded to nearest outside the tensor
// cores (mma_source).  The operators' fragments (hi and lo, per lane)
// are built on the host in FP64 and read from a global table; the data is split on the fly.
//
// Shared memory holds the tiles right-hand side major: in each buffer the tiles of
// right-hand side r start r * rs floats after those of right-hand side 0, with rs = 4
// (mod 32) floats, so that a warp's fragment loads (lanes: 8 right-hand sides x 4 rows
// of k) and stores (8 rows x 4 pairs of right-hand sides) touch 32 distinct banks for any
// odd element stride of the pass's axis.  Inputs and outputs move as runs of tiles per
// right-hand side (cp.async.bulk), as in level_kernel.
//
// Compared with level_kernel's paired FP32 multiply-adds, which skip the unit columns of
// W(delta) and apply diag(phi) per lane, the dense real operator costs (2P)^2 real MACs per
// column for each of the three products; the tensor path is an alternative that the
// autotuner may pick per plan.
#pragma once

#include "level.cuh"

namespace bfly {

constexpr int kTcRhs = 8;  // right-hand sides per work item: the N of m16n8k8

template <int D, int P>
struct TcShape {
  static constexpr int PD = ipow(P, D);
  static constexpr int TS = tile_stride<float>(PD);  // complex elements per stored tile
  static constexpr int FIB = PD / P;
  static constexpr int MT = (2 * P + 15) / 16;  // m16 tiles of the real operator's rows
  static constexpr int KT = (2 * P + 7) / 8;    // k8 steps of its columns
  static constexpr size_t tile_bytes = (size_t)TS * sizeof(float2);  // one right-hand side
  // floats between the tiles of consecutive right-hand sides in a buffer of `cap` tiles
  __host__ __device__ static int rhs_stride(int cap) {
    const int f = cap * TS * 2;
    return f + (((4 - f) % 32) + 32) % 32;
  }
  static constexpr int NSCR = D == 3 ? 2 : 1;
  static size_t bytes(const ChunkCaps &c) {
    return 64 + 2 * (size_t)c.meta_bytes +
           (2 * (size_t)rhs_stride(c.cap0) + NSCR * (size_t)rhs_stride(c.cap1)) * kTcRhs * sizeof(float);
  }
};

// Per-lane A fragments of the real operators, [adjoint][op][mt][kt][hi, lo][lane]
// (a0..a3 of m16n8k8 .row), written once per device and p (init_operators).
static __device__ float4 g_tc_frag[2 * 4 * ((2 * BFLY_P + 15) / 16) * ((2 * BFLY_P + 7) / 8) * 2 * 32];

__device__ __forceinline__ unsigned tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const float4 &a, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(a.z)),
        "r"(__float_as_uint(a.w)), "r"(b0), "r"(b1));
}

template <int D, int P>
struct TcFrag {
  float4 hi[TcShape<D, P>::MT][TcShape<D, P>::KT], lo[TcShape<D, P>::MT][TcShape<D, P>::KT];
};

template <int D, int P, bool ADJ>
__device__ __forceinline__ void load_frag(TcFrag<D, P> &f, int op, int lane) {
  constexpr int MT = TcShape<D, P>::MT, KT = TcShape<D, P>::KT;
  const float4 *t = g_tc_frag + ((size_t)(ADJ ? 4 : 0) + op) * MT * KT * 2 * 32;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      f.hi[mt][kt] = __ldg(t + ((mt * KT + kt) * 2 + 0) * 32 + lane);
      f.lo[mt][kt] = __ldg(t + ((mt * KT + kt) * 2 + 1) * 32 + lane);
    }
}

// R(C) X for one source fibre: X points at element 0 of the fibre of right-hand side 0
// (floats, interleaved re, im), element l of right-hand side r at X[r * rs + 2 l SK + c].
// Lane (g, t4) = (lane / 4, lane % 4) holds the B fragment rows k = 8 kt + t4 and
// 8 kt + t4 + 4 of column (right-hand side) g.
// The MMAs' own accumulation is not rounded to nearest: with every product chained into
// one accumulator the sweep's error was 2e-6 relative on a curve (FP32 multiply-adds:
// 5e-7), which a CPU model that truncates every MMA result toward zero reproduces; the
// truncation is relative to the accumulated value.  So only the small correction
// products (R_lo X_hi, R_hi X_lo) accumulate in the MMAs' chain (`corr`); each k-step's
// main product R_hi X_hi is an MMA of its own (from zero), repeated from minus its result
// to recover what the truncation dropped, and both are added to `acc` in FP32 with
// rounding to nearest (four MMAs per k-step).
template <int D, int P, int SK>
__device__ __forceinline__ void mma_source(float (&acc)[TcShape<D, P>::MT][4], float (&corr)[TcShape<D, P>::MT][4],
                                           const TcFrag<D, P> &f, const float *X, int rs, bool col_on, int g,
                                           int t4) {
  constexpr int MT = TcShape<D, P>::MT, KT = TcShape<D, P>::KT;
  const float *Xg = X + (size_t)g * rs + (t4 & 1);
#pragma unroll
  for (int kt = 0; kt < KT; ++kt) {
    const int l0 = 4 * kt + (t4 >> 1), l1 = l0 + 2;
    const float x0 = (col_on && l0 < P) ? Xg[2 * l0 * SK] : 0.0f;
    const float x1 = (col_on && l1 < P) ? Xg[2 * l1 * SK] : 0.0f;
    const unsigned h0 = tf32_rna(x0), h1 = tf32_rna(x1);
    const unsigned r0 = tf32_rna(x0 - __uint_as_float(h0)), r1 = tf32_rna(x1 - __uint_as_float(h1));
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      mma_tf32(corr[mt], f.lo[mt][kt], h0, h1);
      mma_tf32(corr[mt], f.hi[mt][kt], r0, r1);
      float main[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      mma_tf32(main, f.hi[mt][kt], h0, h1);
      // the same product from -main: what the truncation of `main` dropped
      float res[4] = {-main[0], -main[1], -main[2], -main[3]};
      mma_tf32(res, f.hi[mt][kt], h0, h1);
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[mt][i] += main[i] + res[i];
    }
  }
}

// Pass K of the consumer warps on the tensor cores.  Work unit: one fibre of one item for
// the item's (up to eight) right-hand sides; units of two-source items count twice, and
// the warps split the pass's work evenly (units in program order: two-source items first).
template <int D, int P, int K, bool ADJ>
__device__ __forceinline__ void run_pass_tc(const Item *items, int n_items, int n_two, const float *src,
                                            int src_rs, float *dst, int dst_rs, int nr, int warp, int lane) {
  using S = TcShape<D, P>;
  constexpr int FIB = S::FIB, TS = S::TS, MT = S::MT;
  constexpr int SK = ipow(P, D - 1 - K);
  const int nu = n_items * FIB, nu2 = n_two * FIB;
  const int total = nu + nu2;
  const int per = (total + kConsumerWarps - 1) / kConsumerWarps;
  const int w0 = min(total, warp * per), w1 = min(total, w0 + per);
  auto first_unit = [&](int w) { return w <= 2 * nu2 ? (w + 1) / 2 : w - nu2; };
  const int u0 = first_unit(w0), u1 = first_unit(w1);
  const int g = lane >> 2, t4 = lane & 3;
  const bool col_on = g < nr;
  TcFrag<D, P> f0, f1;
  int cur0 = -1, cur1 = -1;
#pragma unroll 1
  for (int u = u0; u < u1; ++u) {
    const int ti = u / FIB, fb = u - ti * FIB;
    __builtin_assume(fb >= 0 && fb < FIB);
    const Item it = items[ti];
    const int base = (fb / SK) * SK * P + (fb % SK);
    const int op0 = it.ops & 3, op1 = (it.ops >> 2) & 3;
    if (op0 != cur0) {
      load_frag<D, P, ADJ>(f0, op0, lane);
      cur0 = op0;
    }
    float acc[MT][4], corr[MT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[mt][i] = corr[mt][i] = 0.0f;
    mma_source<D, P, SK>(acc, corr, f0, src + ((size_t)it.src0 * TS + base) * 2, src_rs, col_on, g, t4);
    if (u < nu2) {
      if (op1 != cur1) {
        load_frag<D, P, ADJ>(f1, op1, lane);
        cur1 = op1;
      }
      mma_source<D, P, SK>(acc, corr, f1, src + ((size_t)it.src1 * TS + base) * 2, src_rs, col_on, g, t4);
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[mt][i] += corr[mt][i];
    // D fragment: rows 16 mt + g (+ 8) = 2 m + c, columns (right-hand sides) 2 t4, 2 t4 + 1
    float *Y = dst + ((size_t)it.dst * TS + base) * 2;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = 16 * mt + g + 8 * h, m = row >> 1, c = row & 1;
        if (m < P) {
          const int r = 2 * t4;
          if (r < nr) Y[(size_t)r * dst_rs + 2 * m * SK + c] = acc[mt][2 * h];
          if (r + 1 < nr) Y[(size_t)(r + 1) * dst_rs + 2 * m * SK + c] = acc[mt][2 * h + 1];
        }
      }
  }
}

// Pass K of the consumer warps with paired FP32 multiply-adds on the same right-hand-side
// grouped layout (BFLY_FLAG_RHS_GROUPS): a 32-lane step takes four fibres x the eight
// right-hand sides of the group (lane = 8 * fibre + right-hand side), each lane applying
// the factored operators to its fibre exactly as level_kernel's run_pass does (the same
// multiply-adds in the same order, so the results equal level_kernel's).  With the
// right-hand sides rs = 4 (mod 32) floats apart, the two fibres of a half-warp fall on
// disjoint banks whenever their element offsets differ in parity (consecutive fibres of a
// tile), where level_kernel's lanes (one fibre each, tile slots data dependent) conflict
// on about half of the wavefronts; the chunk's program and runs are read once per eight
// right-hand sides.
template <int D, int P, int K, bool ADJ>
__device__ __forceinline__ void run_pass_rg(const Item *items, int n_items, int n_two, const float *src,
                                            int src_rs, float *dst, int dst_rs, int nr, int warp, int lane) {
  using C = float2;
  using S = TcShape<D, P>;
  constexpr int FIB = S::FIB, TS = S::TS;
  constexpr int SK = ipow(P, D - 1 - K);
  constexpr int FPS = 32 / kTcRhs;  // fibres per step
  const int nfib = n_items * FIB, nfib2 = n_two * FIB;
  const int steps = (nfib + FPS - 1) / FPS, steps2 = (nfib2 + FPS - 1) / FPS;
  const int total = steps + steps2;
  const int per = (total + kConsumerWarps - 1) / kConsumerWarps;
  const int w0 = min(total, warp * per), w1 = min(total, w0 + per);
  auto first_step = [&](int w) { return w <= 2 * steps2 ? (w + 1) / 2 : w - steps2; };
  const int s0 = first_step(w0), s1 = first_step(w1);
  const int rr = lane & (kTcRhs - 1), fsub = lane / kTcRhs;
  if (rr >= nr) return;  // a partial group: these lanes have no right-hand side
  const C *srcr = reinterpret_cast<const C *>(src + (size_t)rr * src_rs);
  C *dstr = reinterpret_cast<C *>(dst + (size_t)rr * dst_rs);
#pragma unroll 1
  for (int st = s0; st < s1; ++st) {
    const int fl = st * FPS + fsub;
    if (fl >= nfib) continue;
    const int ti = fl / FIB, f = fl - ti * FIB;
    __builtin_assume(f >= 0 && f < FIB);
    const Item it = items[ti];
    const int base = (f / SK) * SK * P + (f % SK);
    C y[P];
#pragma unroll
    for (int m = 0; m < P; ++m) y[m] = make_float2(0.0f, 0.0f);
    const C *X0 = srcr + (size_t)it.src0 * TS + base;
    const bool d0 = (it.ops & 1) != 0, g0 = (it.ops & 2) != 0;
    if (fl < nfib2) {
      const C *X1 = srcr + (size_t)it.src1 * TS + base;
      if constexpr (!ADJ) {
        apply_factored<float, P, SK, ADJ, 0>(g0, X0, y);
        apply_factored<float, P, SK, ADJ, 1>(g0, X1, y);
      } else if (d0) {
        apply_factored<float, P, SK, ADJ, 1>(true, X1, y);
        apply_factored<float, P, SK, ADJ, 1>(false, X0, y);
      } else {
        apply_factored<float, P, SK, ADJ, 0>(true, X1, y);
        apply_factored<float, P, SK, ADJ, 0>(false, X0, y);
      }
    } else if (d0) {
      apply_factored<float, P, SK, ADJ, 1>(g0, X0, y);
    } else {
      apply_factored<float, P, SK, ADJ, 0>(g0, X0, y);
    }
    C *Y = dstr + (size_t)it.dst * TS + base;
#pragma unroll
    for (int m = 0; m < P; ++m) Y[m * SK] = y[m];
  }
}

template <bool MMA, int D, int P, int K, bool ADJ>
__device__ __forceinline__ void run_pass_group(const Item *items, int n_items, int n_two, const float *src,
                                               int src_rs, float *dst, int dst_rs, int nr, int warp, int lane) {
  if constexpr (MMA)
    run_pass_tc<D, P, K, ADJ>(items, n_items, n_two, src, src_rs, dst, dst_rs, nr, warp, lane);
  else
    run_pass_rg<D, P, K, ADJ>(items, n_items, n_two, src, src_rs, dst, dst_rs, nr, warp, lane);
}

// The persistent, warp-specialised kernel of level_kernel with work items (chunk, group
// of eight right-hand sides): the producer copies every right-hand side of the group run
// by run, the consumers run the passes on the tensor cores (MMA) or with paired FP32
// multiply-adds (run_pass_rg).
template <int D, int P, bool ADJ, bool MMA>
__global__ void __launch_bounds__(kLevelThreads, MMA ? 2 : 3) level_tc_kernel(const LevelArgs a) {
  using S = TcShape<D, P>;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *ptr = smem;
  uint64_t *full = reinterpret_cast<uint64_t *>(ptr);  // full[2], staged[2]
  uint64_t *staged = full + 2;
  int *end_it = reinterpret_cast<int *>(full + 4);  // end_it[0]; end_it[1 + s]: slot s's group size
  ptr += 64;
  unsigned char *meta0 = ptr;
  ptr += 2 * (size_t)a.meta_bytes;
  const int rs0 = S::rhs_stride(a.cap0), rs1 = S::rhs_stride(a.cap1);
  // slot s: input buffer at slot0 + s * kTcRhs * rs0; scratch s at
  // scr0 + (s mod NSCR) * kTcRhs * rs1 (floats)
  float *slot0 = reinterpret_cast<float *>(ptr);
  float *scr0 = slot0 + 2 * (size_t)kTcRhs * rs0;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&staged[0], 1);
    mbar_init(&staged[1], 1);
    *end_it = 0x7fffffff;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  pdl_trigger();

  const unsigned char *gin = reinterpret_cast<const unsigned char *>(a.in);
  unsigned char *gout = reinterpret_cast<unsigned char *>(a.out);
  const int ngroups = (a.nrhs + kTcRhs - 1) / kTcRhs;

  if (warp == kConsumerWarps) {
    // ---------------- producer warp: work items w = chunk * ngroups + group
    const long long total = (long long)a.nchunks * ngroups;
    int slot_it[2] = {-1, -1};
    long long slot_w[2] = {-1, -1};
    int phase_it[2] = {-1, -1};
    bool failed = false, waited = false;
    auto wait_staged = [&](int s, int prev) -> bool {
      const bool ok = mbar_wait(&staged[s], (prev >> 1) & 1, a.wait_limit);
      return __all_sync(0xffffffffu, ok);
    };
    auto write_back = [&](int s, long long w) {
      const unsigned char *meta_s = meta0 + (size_t)s * a.meta_bytes;
      const int32_t *hdr = reinterpret_cast<const int32_t *>(meta_s);
      const int NP = hdr[0], n_oruns = hdr[2];
      int n_items = 0;
      for (int j = 0; j < NP; ++j) n_items += hdr[4 + j];
      const Run *oruns = reinterpret_cast<const Run *>(meta_s + kBlobHeader + (size_t)n_items * sizeof(Item));
      // the last pass wrote the input buffer (odd pass) or the scratch buffer (even)
      const bool in_buf = ((NP - 1) & 1) != 0;
      const float *stage_f = in_buf ? slot0 + (size_t)s * kTcRhs * rs0 : scr0 + (size_t)(s % S::NSCR) * kTcRhs * rs1;
      const int st_rs = in_buf ? rs0 : rs1;
      unsigned char *obase = gout;
      int64_t orhs = a.out_rhs;
      if (a.entries) {
        const BatchEntry &be = a.entries[w / ngroups];
        obase = reinterpret_cast<unsigned char *>(be.out);
        orhs = be.out_rhs;
      }
      const int r0 = (int)(w % ngroups) * kTcRhs, nr = min(kTcRhs, a.nrhs - r0);
      for (int j = lane; j < n_oruns * nr; j += 32) {
        const int rr = j / n_oruns;
        const Run rn = oruns[j - rr * n_oruns];
        const unsigned char *stage = reinterpret_cast<const unsigned char *>(stage_f + (size_t)rr * st_rs);
        unsigned char *rout = obase + (size_t)(r0 + rr) * orhs * sizeof(float2);
        bulk_s2g(rout + (size_t)rn.start * S::tile_bytes, stage + (size_t)rn.slot * S::tile_bytes,
                 (unsigned)(rn.count * S::tile_bytes));
      }
      bulk_commit();
      bulk_wait_read();
      __syncwarp();
    };
    int it = 0;
    for (;; ++it) {
      const int s = it & 1;
      const bool wb = slot_it[s] >= 0;
      if (wb && !wait_staged(s, slot_it[s])) {
        failed = true;
        break;
      }
      long long w = blockIdx.x;
      if (it > 0 && lane == 0) w = (long long)gridDim.x + (long long)atomicAdd(a.sched, 1ull);
      if (wb) {
        write_back(s, slot_w[s]);
        slot_it[s] = -1;
      }
      w = __shfl_sync(0xffffffffu, w, 0);
      if (w >= total) {
        if (lane == 0) {
          *end_it = it;
          mbar_arrive(&full[s]);
        }
        phase_it[s] = it;
        __syncwarp();
        break;
      }
      const long long ch = w / ngroups;
      const int r0 = (int)(w % ngroups) * kTcRhs, nr = min(kTcRhs, a.nrhs - r0);
      const ChunkDesc cd = a.entries ? a.entries[ch].d : a.chunks[ch];
      const unsigned char *blob = a.entries ? a.entries[ch].blob : a.blob;
      const Run *runs = a.entries ? a.entries[ch].runs : a.runs;
      const unsigned char *ibase = a.entries ? reinterpret_cast<const unsigned char *>(a.entries[ch].in) : gin;
      const int64_t irhs = a.entries ? a.entries[ch].in_rhs : a.in_rhs;
      slot_it[s] = it;
      slot_w[s] = w;
      if (a.inject_stall && it == 0) {
        if (!waited) {
          pdl_wait();
          waited = true;
        }
        continue;
      }
      unsigned char *meta_s = meta0 + (size_t)s * a.meta_bytes;
      float *in_s = slot0 + (size_t)s * kTcRhs * rs0;
      if (lane == 0) {
        end_it[1 + s] = nr;  // read by the consumers after this phase completes
        mbar_arrive_expect_tx(&full[s], (unsigned)(cd.blob_bytes + cd.n_in * nr * (int)S::tile_bytes));
        bulk_g2s(meta_s, blob + cd.blob_off, (unsigned)cd.blob_bytes, &full[s]);
      }
      __syncwarp();
      if (!waited) {
        pdl_wait();
        waited = true;
      }
      for (int j = lane; j < cd.n_runs * nr; j += 32) {
        const int rr = j / cd.n_runs;
        const Run rn = runs[cd.run_off + j - rr * cd.n_runs];
        const unsigned char *rin = ibase + (size_t)(r0 + rr) * irhs * sizeof(float2);
        unsigned char *dst = reinterpret_cast<unsigned char *>(in_s + (size_t)rr * rs0);
        bulk_g2s(dst + (size_t)rn.slot * S::tile_bytes, rin + (size_t)rn.start * S::tile_bytes,
                 (unsigned)(rn.count * S::tile_bytes), &full[s]);
      }
      phase_it[s] = it;
    }
    const int sl = (it + 1) & 1;
    if (!failed && slot_it[sl] >= 0) {
      if (wait_staged(sl, slot_it[sl])) write_back(sl, slot_w[sl]);
      else failed = true;
    }
    if (!waited) pdl_wait();
    if (failed && lane == 0) atomicOr(a.status, 1);
    for (int s = 0; s < 2; ++s) {
      const bool ok = phase_it[s] < 0 || mbar_wait(&full[s], (phase_it[s] >> 1) & 1, a.wait_limit);
      if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(a.status, 2);
    }
    bulk_wait_all();
    if (lane == 0) {
      __threadfence();
      if (atomicAdd(&a.sched[1], 1ull) == (unsigned long long)gridDim.x - 1) {
        atomicExch(&a.sched[0], 0ull);
        atomicExch(&a.sched[1], 0ull);
      }
    }
    return;
  }

  // ---------------- consumer warps
  pdl_wait();
  for (int it = 0;; ++it) {
    const int s = it & 1, use = it >> 1;
    const bool ok = mbar_wait(&full[s], use & 1, a.wait_limit);
    if (consumer_any(!ok)) {
      if (tid == 0) atomicOr(a.status, 4);
      break;
    }
    if (it == *static_cast<volatile int *>(end_it)) break;
    const unsigned char *meta_s = meta0 + (size_t)s * a.meta_bytes;
    float *in_s = slot0 + (size_t)s * kTcRhs * rs0;
    float *scr = scr0 + (size_t)(s % S::NSCR) * kTcRhs * rs1;
    const int32_t *hdr = reinterpret_cast<const int32_t *>(meta_s);
    const int NP = hdr[0];
    const Item *ip = reinterpret_cast<const Item *>(meta_s + kBlobHeader);
    // right-hand sides of this item's group (written by the producer before the slot's
    // phase began, so ordered by the mbarrier like the copied data)
    const int nr = *reinterpret_cast<const volatile int *>(end_it + 1 + s);
    for (int j = 0; j < NP; j += D) {
      if (j > 0) consumer_sync();
      run_pass_group<MMA, D, P, 0, ADJ>(ip, hdr[4 + j], hdr[4 + kMaxPasses + j], (j & 1) ? scr : in_s, (j & 1) ? rs1 : rs0,
                                (j & 1) ? in_s : scr, (j & 1) ? rs0 : rs1, nr, warp, lane);
      ip += hdr[4 + j];
      consumer_sync();
      run_pass_group<MMA, D, P, 1, ADJ>(ip, hdr[5 + j], hdr[5 + kMaxPasses + j], (j & 1) ? in_s : scr, (j & 1) ? rs0 : rs1,
                                (j & 1) ? scr : in_s, (j & 1) ? rs1 : rs0, nr, warp, lane);
      ip += hdr[5 + j];
      if constexpr (D == 3) {
        consumer_sync();
        run_pass_group<MMA, D, P, (D == 3 ? 2 : 0), ADJ>(ip, hdr[6 + j], hdr[6 + kMaxPasses + j], (j & 1) ? scr : in_s,
                                                 (j & 1) ? rs1 : rs0, (j & 1) ? in_s : scr, (j & 1) ? rs0 : rs1, nr,
                                                 warp, lane);
        ip += hdr[6 + j];
      }
    }
    fence_async_shared();
    consumer_sync();
    if (tid == 0) mbar_arrive(&staged[s]);
  }
}

}  // namespace bfly
