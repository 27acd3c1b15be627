// Recursive step of the butterfly (Sec. 2.2 step 3, Fig. 1): one launch per step of up to
// three consecutive stages (2D; one in 3D), or all steps in one launch whose chunks wait
// for the chunks they read (the dataflow launch, flow_producer below).
//
// For every pair (A, B) at stage t the charges are
//     f^{AB} = sum_{c in children(B)} ( (x)_d T^{(alpha_d(A), delta_d(c))} ) f^{A' Bc}
// with A' the parent of A and T the per-axis transfer operators (plan.cpp).  The host
// compiles every step into chunks of units with one item list per pass: pass j applies
// the operator of axis j mod D to at most two source tiles and sums them (the sources
// agree on every bit still to be applied; sum factorisation).  The passes alternate
// between the slot's input buffer and the scratch buffer,
//   inputs --pass 0--> scratch --pass 1--> input slot --pass 2--> scratch ...,
// and the last pass's tiles are written back; in a two-stage step the tiles of the stage
// between the two levels never leave shared memory.  The adjoint sweep runs the same kernel on the adjoint program with the
// conjugate-transposed operators.  A batched launch runs the chunks of many plans (same
// dim, p and precision): a per-chunk entry then names the chunk's buffers.
//
// A persistent block is warp-specialised.  One producer warp walks over the block's
// chunks (times right-hand sides).  For chunk i in slot s = i mod 2 it first writes back
// the outputs of chunk i-2, staged by the consumers in slot s (bulk stores of contiguous
// output runs, cp.async.bulk shared -> global), waits until those stores have read the
// slot, then copies chunk i's metadata blob and input tiles (runs of consecutive 16-byte
// aligned tiles) into the slot with bulk copies completing on the slot's "full" mbarrier.
// The consumer warps wait on "full" and run the passes.  A pass's fibres (two-source
// items first, then ordered by operator) are taken 32 at a time ("steps", one fibre per
// lane), the warps split the pass's work (one unit per source of a step) evenly, and
// every lane of a step computes y = C^{op0} x0 (+ C^{op1} x1) for its fibre.  Each
// operator is applied in its factored form C^{(gamma,delta)} = W(delta) diag(phi_gamma):
// the lane's own diagonal (phi_0 = 1), then W(delta), whose entries live in constant
// memory and enter the (paired, f32x2) multiply-adds as warp-uniform operands (delta is the same in
// every lane of a step but at most one step per pass, where the two halves run one after
// the other).  Per fibre: P (or 2P) shared-memory loads, P^2 (or 2P^2) complex
// multiply-adds, P stores; one barrier per pass.  The last
// pass stages its tiles in the slot; the consumers then signal
// the slot's "staged" mbarrier and go on with the other slot, so that the write-back and
// the next copies overlap their compute.  Every mbarrier wait gives up after a clock
// budget, sets the status word and leaves the loop together with its peers; the producer
// then waits (again bounded) for the copies it issued before the block exits.
#pragma once

#include "common.cuh"

namespace bfly {

template <typename R>
__host__ __device__ constexpr int tile_stride(int pd) {
  // complex elements per stored tile: a multiple of 16 bytes
  return sizeof(R) == 4 ? (pd + 1) & ~1 : pd;
}

constexpr int kConsumerWarps = 7;  // + 1 producer: 8 warps, two per SM sub-partition
static_assert(kConsumerWarps == kProgramWarps, "the chunk programs are balanced for this count");
constexpr int kLevelThreads = (kConsumerWarps + 1) * 32;
constexpr int kLevelBlocksPerSm = 4;

template <typename R, int D, int P>
struct LevelShape {
  using C = typename Cx<R>::T;
  static constexpr int Q = P - 1;
  static constexpr int NOPS = 4;  // C^{(gamma, delta)}, op = gamma*2 + delta
  static constexpr int PD = ipow(P, D);
  static constexpr int TS = tile_stride<R>(PD);
  static constexpr int FIB = PD / P;  // fibres of one tile along one axis
  static constexpr size_t tile_bytes = (size_t)TS * sizeof(C);
  static int meta_bytes(int cap0, int cap1, int max_out) {
    // header, an item (8 bytes) per pass tile, one run (8 bytes) per output, padding.  In
    // 2D a step has up to three levels (passes alternately into the scratch and input
    // buffers, the last into the staged outputs); in 3D one
    const int items = (D == 2 ? 3 * cap1 + 2 * cap0 : cap1 + cap0) + max_out;
    return (kBlobHeader + 8 * items + 8 * max_out + 15) & ~15;
  }
  // 4 mbarriers | 2 metadata slots | 2 input buffers | scratch (2 in 3D, where a
  // one-level step stages its outputs there)
  static constexpr int NSCR = D == 3 ? 2 : 1;
  static size_t bytes(const ChunkCaps &c) {
    size_t b = 64;
    b += 2 * (size_t)c.meta_bytes;
    return b + (2 * (size_t)c.cap0 + NSCR * (size_t)c.cap1) * tile_bytes;
  }
};

// ---- PTX wrappers: mbarrier and 1D bulk copies (sm_90+)
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// Waits for the phase of `bar` with the given parity to complete; false after `limit`
// clock cycles.  Between polls the warp sleeps (growing to `max_sleep_ns`), so that a
// waiting warp leaves the issue slots of its SM sub-partition to the computing warps.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit,
                                          unsigned max_sleep_ns = 256) {
  const unsigned a = smem_addr(bar);
  const long long t0 = clock64();
  unsigned ns = 8;
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
    __nanosleep(ns);
    if (ns < max_sleep_ns) ns *= 2;
  }
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Cross-block signalling of the dataflow launch: the bulk stores of an item's outputs
// (async proxy) complete, a proxy fence orders them with the generic proxy, a release
// fence and a store publish the item's flag; a reader that sees the flag takes an acquire
// fence and fences the async proxy before its bulk copies of those outputs.
__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned *p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_release_gpu() { asm volatile("fence.release.gpu;\n" ::: "memory"); }
__device__ __forceinline__ void fence_acquire_gpu() { asm volatile("fence.acquire.gpu;\n" ::: "memory"); }
// Adds `bytes` to the transaction count of the current phase of `bar` (no arrival).
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;\n" ::"r"(kConsumerWarps * 32) : "memory");
}
// Barrier over the consumer warps that also returns whether any of them passed `v`.
__device__ __forceinline__ bool consumer_any(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 2, %2, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)v), "r"(kConsumerWarps * 32)
      : "memory");
  return r != 0;
}

// The factors of the transfer operators of this translation unit's p (BFLY_P), both
// directions: c_w[adjoint][delta][m][l] (W(delta), or W(delta)^H) and
// c_phi[adjoint][delta][l] (phi_1, or its conjugate).  The same for every plan of that p,
// written once per device (init_operators).
#ifndef BFLY_P
#error "level.cuh is compiled once per p, with BFLY_P defined"
#endif
// FP32 entries are stored packed as (re, re, -im, im): a complex multiply-add is then two
// paired multiply-adds (fma.rn.f32x2), (re, re) * (x.x, x.y) + (-im, im) * (x.y, x.x),
// with the same roundings and order as the four scalar ones.
static __constant__ float4 c_w32[2][2][BFLY_P][BFLY_P];
static __constant__ float4 c_phi32[2][2][BFLY_P];
static __constant__ double2 c_w64[2][2][BFLY_P][BFLY_P];
static __constant__ double2 c_phi64[2][2][BFLY_P];

template <bool ADJ, int DL>
__device__ __forceinline__ float4 w_packed(int m, int l) { return c_w32[ADJ][DL][m][l]; }
template <bool ADJ, int DL>
__device__ __forceinline__ float4 phi_packed(int l) { return c_phi32[ADJ][DL][l]; }
template <bool ADJ, int DL>
__device__ __forceinline__ double2 w_entry64(int m, int l) { return c_w64[ADJ][DL][m][l]; }
template <bool ADJ, int DL>
__device__ __forceinline__ double2 phi_entry64(int l) { return c_phi64[ADJ][DL][l]; }

// acc + c x for a packed constant c = (re, re, -im, im)
__device__ __forceinline__ float2 cmac2(float4 c, float2 x, float2 acc) {
  acc = __ffma2_rn(make_float2(c.x, c.y), x, acc);
  return __ffma2_rn(make_float2(c.z, c.w), make_float2(x.y, x.x), acc);
}
__device__ __forceinline__ float2 cmul2(float4 c, float2 x) {
  return cmac2(c, x, make_float2(0.0f, 0.0f));
}

// y += C^{(gamma, DL)} x for one fibre, x_l = X[l * SK]: forward W(DL) (phi_gamma o x),
// adjoint conj(phi_gamma) o (W(DL)^H x).  The loops are unrolled, so every entry of W and
// phi has a compile-time address and is read as a constant-bank operand.
// One source of a lane's fibre, x = X[l * SK]:
//   forward  y += W(DL) (phi_gamma o x)
//   adjoint  y += W(DL)^H x, then, for gamma = 1, y = conj(phi_1) o y (the caller takes
//            the gamma = 1 source of an item first, so that the scaling applies to that
//            source alone and no second accumulator is needed).
// Half of the child grid points lie on parent grid nodes: tau_l = (DL q + l)/(2q) is the
// node m' = (DL q + l)/2 when DL q + l is even (q = P - 1 is even), and there the
// Lagrange weights are the unit vector w(tau_l) = e_{m'} (interpolation property).  Those
// columns of W (rows of W^H) cost one addition instead of P multiply-adds; only the
// other entries are read.  The loops are unrolled: the node tests fold at compile time
// and every remaining entry of W and phi has a compile-time address in constant memory.
// (Two fibres per lane sharing each entry measured 15-29 % slower: larger unrolled
// bodies and register pressure.)
template <typename R, int P, int SK, bool ADJ, int DL>
__device__ __forceinline__ void apply_factored(bool gamma, const typename Cx<R>::T *X,
                                               typename Cx<R>::T (&y)[P]) {
  using C = typename Cx<R>::T;
  constexpr int Q = P - 1;
  static_assert(Q % 2 == 0, "odd p: the child grid's even points are parent nodes");
  C x[P];
#pragma unroll
  for (int l = 0; l < P; ++l) x[l] = X[l * SK];
  if constexpr (!ADJ) {
    if (gamma) {
#pragma unroll
      for (int l = 0; l < P; ++l) {
        if constexpr (sizeof(R) == 4)
          x[l] = cmul2(phi_packed<ADJ, DL>(l), x[l]);
        else
          x[l] = cmul(phi_entry64<ADJ, DL>(l), x[l]);
      }
    }
    // l outer, m inner: P independent multiply-add chains in flight
#pragma unroll
    for (int l = 0; l < P; ++l) {
      if (((DL * Q + l) & 1) == 0) {  // a parent node: a unit column
        y[(DL * Q + l) >> 1] = cadd(y[(DL * Q + l) >> 1], x[l]);
      } else {
#pragma unroll
        for (int m = 0; m < P; ++m) {
          if constexpr (sizeof(R) == 4)
            y[m] = cmac2(w_packed<ADJ, DL>(m, l), x[l], y[m]);
          else
            y[m] = cfma(w_entry64<ADJ, DL>(m, l), x[l], y[m]);
        }
      }
    }
  } else {
    // W^H: the rows of the parent nodes are unit rows
#pragma unroll
    for (int r = 0; r < P; ++r)
      if (((DL * Q + r) & 1) == 0) y[r] = cadd(y[r], x[(DL * Q + r) >> 1]);
#pragma unroll
    for (int l = 0; l < P; ++l)
#pragma unroll
      for (int r = 0; r < P; ++r) {
        if (((DL * Q + r) & 1) == 0) continue;
        if constexpr (sizeof(R) == 4)
          y[r] = cmac2(w_packed<ADJ, DL>(r, l), x[l], y[r]);
        else
          y[r] = cfma(w_entry64<ADJ, DL>(r, l), x[l], y[r]);
      }
    if (gamma) {
#pragma unroll
      for (int m = 0; m < P; ++m) {
        if constexpr (sizeof(R) == 4)
          y[m] = cmul2(phi_packed<ADJ, DL>(m), y[m]);
        else
          y[m] = cmul(phi_entry64<ADJ, DL>(m), y[m]);
      }
    }
  }
}

// Pass K, warp `warp` of the consumers.  The pass's fibres (n_items * P^(D-1), item by
// item, the n_two two-source items first) are taken 32 at a time ("steps", one fibre per
// lane); a step costs one unit of work per source, and the warps split the work evenly.
// Each lane computes y = C^{op0} x0 (+ C^{op1} x1) along axis K for its fibre with its
// item's operators and stores it to the item's destination tile (every destination of a
// pass is written by exactly one item).
template <typename R, int D, int P, int K, bool ADJ>
__device__ __forceinline__ void run_pass(const Item *items, int n_items, int n_two,
                                         const typename Cx<R>::T *src, typename Cx<R>::T *dst,
                                         int warp, int lane) {
  using C = typename Cx<R>::T;
  using S = LevelShape<R, D, P>;
  constexpr int FIB = S::FIB, TS = S::TS;
  constexpr int SK = ipow(P, D - 1 - K);  // element stride of axis K
  const int nfib = n_items * FIB, nfib2 = n_two * FIB;
  const int steps = (nfib + 31) / 32, steps2 = (nfib2 + 31) / 32;  // steps2: with a two-source fibre
  const int total = steps + steps2;
  const int per = (total + kConsumerWarps - 1) / kConsumerWarps;
  const int w0 = min(total, warp * per), w1 = min(total, w0 + per);
  // the first step whose work starts at or after w: 2s for s < steps2, then steps2 + s
  auto first_step = [&](int w) { return w <= 2 * steps2 ? (w + 1) / 2 : w - steps2; };
  const int s0 = first_step(w0), s1 = first_step(w1);
#pragma unroll 1
  for (int st = s0; st < s1; ++st) {
    const int fl = st * 32 + lane;
    if (fl >= nfib) continue;
    const int ti = fl / FIB, f = fl - ti * FIB;
    __builtin_assume(f >= 0 && f < FIB);  // the fibre's offsets below then need no division
    const Item it = items[ti];
    const int base = (f / SK) * SK * P + (f % SK);
    C y[P];
#pragma unroll
    for (int m = 0; m < P; ++m) y[m] = cmk((R)0, (R)0);
    const C *X0 = src + (size_t)it.src0 * TS + base;
    const bool d0 = (it.ops & 1) != 0, g0 = (it.ops & 2) != 0;
    if (fl < nfib2) {
      // two sources: forward, the delta = 0 and delta = 1 children of the same gamma;
      // adjoint, the gamma = 0 and gamma = 1 children of the same delta (gamma = 1
      // first, so that its scaling applies to it alone)
      const C *X1 = src + (size_t)it.src1 * TS + base;
      if constexpr (!ADJ) {
        apply_factored<R, P, SK, ADJ, 0>(g0, X0, y);
        apply_factored<R, P, SK, ADJ, 1>(g0, X1, y);
      } else if (d0) {
        apply_factored<R, P, SK, ADJ, 1>(true, X1, y);
        apply_factored<R, P, SK, ADJ, 1>(false, X0, y);
      } else {
        apply_factored<R, P, SK, ADJ, 0>(true, X1, y);
        apply_factored<R, P, SK, ADJ, 0>(false, X0, y);
      }
    } else if (d0) {
      apply_factored<R, P, SK, ADJ, 1>(g0, X0, y);
    } else {
      apply_factored<R, P, SK, ADJ, 0>(g0, X0, y);
    }
    C *Y = dst + (size_t)it.dst * TS + base;
#pragma unroll
    for (int m = 0; m < P; ++m) Y[m * SK] = y[m];
  }
}

// Producer warp of a dataflow launch (LevelArgs::deps set: the chunks of every step of
// a sweep in one launch).  Items come from the work counter in order, so that a block
// only ever waits for items that running blocks hold (the grid's blocks need not all be
// resident at once: blocks of kernels queued after this one may take the places of some).
// An item is taken only when its slot is free (taking it one iteration ahead, to hide the
// counter's latency, measured slower: the items in flight then reach further ahead of the
// published ones, and more of them wait).  Iteration it, slot s = it mod 2:
//   1. wait for the consumers to finish iteration it-2, take the item (the counter's
//      latency overlaps the stores of that iteration's outputs); publish the written
//      items (flag = the launch's epoch) once the counter comes near the first item that
//      reads one of them (first_use), until then their stores complete unobserved;
//   2. copy the item's program; if one of its sources is not yet published, first publish
//      everything this block holds (the outputs the consumers are computing included), then
//      wait (bounded) for the sources: the lowest unfinished item then always has its
//      sources, and the launch makes progress;
//   3. copy the item's inputs.
// Publishing waits for the block's stores to land and takes one release fence for all the
// items it publishes; items that no later item reads are never published.
constexpr int kFlowPending = 16;  // written items a block keeps unpublished at most
template <typename R, int D, int P>
__device__ __forceinline__ void flow_producer(const LevelArgs &a, uint64_t *full, uint64_t *staged, int *end_it,
                                              unsigned char *meta0, typename Cx<R>::T *slot0,
                                              typename Cx<R>::T *scr0, int lane) {
  using C = typename Cx<R>::T;
  using S = LevelShape<R, D, P>;
  constexpr int TS = S::TS;
  const int total = a.nchunks * a.nrhs;  // below 2^31 (checked by the plan)
  int slot_it[2] = {-1, -1};       // iteration whose outputs slot s holds, -1: none
  int slot_w[2] = {-1, -1};        // its work item
  int phase_it[2] = {-1, -1};      // last iteration that completes a phase of full[s]
  // written, unpublished items (lane j holds the j-th) and the smallest first_use among them
  int pend_w = -1, n_pend = 0, pend_due = 0x7fffffff;
  bool failed = false;
  // the counter, the flags and every input follow the predecessor grid
  pdl_wait();
  const unsigned epoch = ld_acquire(a.epoch) + 1u;
  auto publish_all = [&]() {
    if (n_pend == 0) return;
    bulk_wait_all();  // the stores have landed
    fence_async_global();
    __syncwarp();
    fence_release_gpu();
    if (lane < n_pend) st_relaxed(&a.flags[pend_w], epoch);
    n_pend = 0;
    pend_due = 0x7fffffff;
    __syncwarp();
  };
  auto wait_staged = [&](int s, int prev) -> bool {
    const bool ok = mbar_wait(&staged[s], (prev >> 1) & 1, a.wait_limit);
    return __all_sync(0xffffffffu, ok);
  };
  // issues the stores of the outputs staged in slot s by item w (published later)
  auto write_back = [&](int s, int w) {
    if (n_pend == kFlowPending) publish_all();
    const unsigned char *meta_s = meta0 + (size_t)s * a.meta_bytes;
    const int32_t *hdr = reinterpret_cast<const int32_t *>(meta_s);
    const int NP = hdr[0], n_oruns = hdr[2];
    int n_items = 0;
    for (int j = 0; j < NP; ++j) n_items += hdr[4 + j];
    const Run *oruns = reinterpret_cast<const Run *>(meta_s + kBlobHeader + (size_t)n_items * sizeof(Item));
    const C *stage_t = ((NP - 1) & 1) ? slot0 + (size_t)s * a.cap0 * TS : scr0 + (size_t)(s % S::NSCR) * a.cap1 * TS;
    const unsigned char *stage = reinterpret_cast<const unsigned char *>(stage_t);
    const int e = w / a.nrhs;
    const BatchEntry &be = a.entries[e];
    unsigned char *rout = reinterpret_cast<unsigned char *>(be.out) + (size_t)(w % a.nrhs) * be.out_rhs * sizeof(C);
    for (int j = lane; j < n_oruns; j += 32) {
      const Run rn = oruns[j];
      bulk_s2g(rout + (size_t)rn.start * S::tile_bytes, stage + (size_t)rn.slot * S::tile_bytes,
               (unsigned)(rn.count * S::tile_bytes));
    }
    bulk_commit();
    bulk_wait_read();  // the slot may be refilled after this
    __syncwarp();
    const int fu = a.first_use[e];
    if (fu >= 0) {  // read by a later item
      if (lane == n_pend) pend_w = w;
      ++n_pend;
      if (fu < pend_due) pend_due = fu;
    }
  };
  // the entries whose outputs item w reads, loaded early (their flags are read later):
  // the entry's row {count, sources...} of LevelArgs::deps, lane j holding elements j and
  // 32 + j (-1 past the count)
  auto load_deps = [&](int w, int &d0, int &d1) {
    d0 = d1 = -1;
    if (w >= total) return;
    const int *row = a.deps + (size_t)(w / a.nrhs) * kFlowDepRow;
    d0 = row[lane];
    d1 = row[32 + lane];
  };
  // whether every item whose outputs item w reads carries this launch's epoch
  auto sources_ready = [&](int w, int d0, int d1) -> bool {
    const int r = w % a.nrhs;
    const int count = __shfl_sync(0xffffffffu, d0, 0);
    if (count <= 0) return true;
    bool ok = true;
    if (count < kFlowDepRow) {
      if (lane > 0 && d0 >= 0) ok = ld_relaxed(&a.flags[d0 * a.nrhs + r]) == epoch;
      if (d1 >= 0) ok &= ld_relaxed(&a.flags[d1 * a.nrhs + r]) == epoch;
    } else {
      // more sources than a row holds: the full list
      const int e = w / a.nrhs;
      for (int j = a.dep_off[e] + lane; j < a.dep_off[e + 1]; j += 32)
        ok &= ld_relaxed(&a.flags[a.dep_idx[j] * a.nrhs + r]) == epoch;
    }
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
      // the sources' outputs are visible after the flags, to every lane
      fence_acquire_gpu();
      __syncwarp();
    }
    return ok;
  };
  int w = 0, dep0 = -1, dep1 = -1;
  int it = 0;
  for (;; ++it) {
    const int s = it & 1;
    // 1.
    const bool wb = slot_it[s] >= 0;
    if (wb && !wait_staged(s, slot_it[s])) {
      failed = true;
      break;
    }
    int nxt = 0;
    if (lane == 0) nxt = (int)min(atomicAdd(a.sched, 1ull), (unsigned long long)total);
    if (wb) {
      write_back(s, slot_w[s]);
      slot_it[s] = -1;
    }
    w = __shfl_sync(0xffffffffu, nxt, 0);
    // the blocks take about one item each while this one computes one: publish the written
    // items once the counter is within two rounds of the grid of the first reader (before
    // this item's copies: a reader may be waiting)
    if (n_pend > 0 && (long long)w + 2LL * gridDim.x >= (long long)pend_due * a.nrhs) publish_all();
    load_deps(w, dep0, dep1);
    if (w >= total) {
      // no more work: the consumers stop at iteration it (the phase completes without data)
      if (lane == 0) {
        *end_it = it;
        mbar_arrive(&full[s]);
      }
      phase_it[s] = it;
      __syncwarp();
      break;
    }
    const BatchEntry &be = a.entries[w / a.nrhs];
    const ChunkDesc cd = be.d;
    slot_it[s] = it;
    slot_w[s] = w;
    if (a.inject_stall && it == 0) continue;  // test hook: the first item never arrives
    // 2.
    unsigned char *meta_s = meta0 + (size_t)s * a.meta_bytes;
    unsigned char *in_s = reinterpret_cast<unsigned char *>(slot0 + (size_t)s * a.cap0 * TS);
    if (lane == 0) {
      mbar_expect_tx(&full[s], (unsigned)cd.blob_bytes);
      bulk_g2s(meta_s, be.blob + cd.blob_off, (unsigned)cd.blob_bytes, &full[s]);
    }
    __syncwarp();
    bool ready = sources_ready(w, dep0, dep1);
    if (!ready) {
      publish_all();
      const int o = s ^ 1;
      if (slot_it[o] >= 0) {
        if (!wait_staged(o, slot_it[o])) failed = true;
        else write_back(o, slot_w[o]);
        slot_it[o] = -1;
        publish_all();
      }
      // bounded wait (the decision to give up is the warp's, from lane 0's clock)
      const long long t0 = clock64();
      unsigned ns = 32;
      while (!failed) {
        ready = sources_ready(w, dep0, dep1);
        if (ready || __shfl_sync(0xffffffffu, clock64() - t0 > a.wait_limit, 0)) break;
        __nanosleep(ns);
        if (ns < 512) ns *= 2;
      }
      if (!ready) {
        // the consumers stop at this iteration once the program has landed
        if (lane == 0) {
          if (!failed) atomicOr(a.status, 8);
          *end_it = it;
          mbar_arrive(&full[s]);
        }
        slot_it[s] = -1;
        phase_it[s] = it;
        failed = true;
        __syncwarp();
        break;
      }
    }
    // 3.
    fence_async_global();
    if (lane == 0) mbar_arrive_expect_tx(&full[s], (unsigned)(cd.n_in * (int)S::tile_bytes));
    __syncwarp();
    const unsigned char *rin =
        reinterpret_cast<const unsigned char *>(be.in) + (size_t)(w % a.nrhs) * be.in_rhs * sizeof(C);
    for (int j = lane; j < cd.n_runs; j += 32) {
      const Run rn = be.runs[cd.run_off + j];
      bulk_g2s(in_s + (size_t)rn.slot * S::tile_bytes, rin + (size_t)rn.start * S::tile_bytes,
               (unsigned)(rn.count * S::tile_bytes), &full[s]);
    }
    phase_it[s] = it;
  }
  // the outputs of the iteration before the last
  const int sl = (it + 1) & 1;
  if (!failed && slot_it[sl] >= 0) {
    if (wait_staged(sl, slot_it[sl])) write_back(sl, slot_w[sl]);
    else failed = true;
  }
  publish_all();
  if (failed && lane == 0) atomicOr(a.status, 1);
  // copies still in flight land before the block exits
  for (int s = 0; s < 2; ++s) {
    const bool ok = phase_it[s] < 0 || mbar_wait(&full[s], (phase_it[s] >> 1) & 1, a.wait_limit);
    if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(a.status, 2);
  }
  bulk_wait_all();
  if (lane == 0) {
    // the last block done resets the counter and advances the epoch for the next launch
    __threadfence();
    if (atomicAdd(&a.sched[1], 1ull) == (unsigned long long)gridDim.x - 1) {
      atomicExch(&a.sched[0], 0ull);
      atomicExch(&a.sched[1], 0ull);
      atomicAdd(a.epoch, 1u);
    }
  }
}

// FLOW: a dataflow launch (flow_producer drives the copies); else one launch per step.
template <typename R, int D, int P, bool ADJ, bool FLOW>
__global__ void __launch_bounds__(kLevelThreads, kLevelBlocksPerSm) level_kernel(const LevelArgs a) {
  using C = typename Cx<R>::T;
  using S = LevelShape<R, D, P>;
  constexpr int TS = S::TS;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *ptr = smem;
  uint64_t *full = reinterpret_cast<uint64_t *>(ptr);  // full[2], staged[2]
  uint64_t *staged = full + 2;
  int *end_it = reinterpret_cast<int *>(full + 4);  // first iteration without work
  ptr += 64;
  unsigned char *meta0 = ptr;  // slot s at meta0 + s * meta_bytes
  ptr += 2 * (size_t)a.meta_bytes;
  // slot s: input buffer (cap0 tiles) at slot0 + s * cap0 * TS; scratch s (cap1 tiles)
  // at scr0 + (s mod NSCR) * cap1 * TS
  C *slot0 = reinterpret_cast<C *>(ptr);
  C *scr0 = slot0 + 2 * (size_t)a.cap0 * TS;

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
  // The next stage's blocks may be scheduled now: they take the slots of this grid's
  // blocks as these exit and wait for this grid's outputs (pdl_wait) before their copies.
  pdl_trigger();

  const unsigned char *gin = reinterpret_cast<const unsigned char *>(a.in);
  unsigned char *gout = reinterpret_cast<unsigned char *>(a.out);

  if (warp == kConsumerWarps) {
    if constexpr (FLOW) {
      flow_producer<R, D, P>(a, full, staged, end_it, meta0, slot0, scr0, lane);
      return;
    }
    // ---------------- producer warp.  Work items w = chunk * nrhs + rhs, the chunks in
    // decreasing work: block b first takes item b, then the next untaken item of the
    // launch's counter (gridDim.x + a.sched[0]), so that the blocks finish together.
    // Iteration it uses slot it mod 2: write-back of the outputs of iteration it-2, then
    // the copies of the new item.
    const long long total = (long long)a.nchunks * a.nrhs;
    int slot_it[2] = {-1, -1};        // iteration whose outputs slot s holds, -1: none
    long long slot_w[2] = {-1, -1};   // its work item
    int phase_it[2] = {-1, -1};       // last iteration that completes a phase of full[s]
    bool failed = false, waited = false;
    // writes back the outputs staged in slot s by iteration `prev` (item w); false on a
    // timeout
    auto wait_staged = [&](int s, int prev) -> bool {
      const bool ok = mbar_wait(&staged[s], (prev >> 1) & 1, a.wait_limit);
      return __all_sync(0xffffffffu, ok);
    };
    // writes back the outputs staged in slot s by item w (after wait_staged)
    auto write_back = [&](int s, long long w) {
      const unsigned char *meta_s = meta0 + (size_t)s * a.meta_bytes;
      const int32_t *hdr = reinterpret_cast<const int32_t *>(meta_s);
      const int NP = hdr[0], n_oruns = hdr[2];
      int n_items = 0;
      for (int j = 0; j < NP; ++j) n_items += hdr[4 + j];
      const Run *oruns = reinterpret_cast<const Run *>(meta_s + kBlobHeader + (size_t)n_items * sizeof(Item));
      // the last pass wrote the input buffer (odd pass) or the scratch buffer (even)
      const C *stage_t = ((NP - 1) & 1) ? slot0 + (size_t)s * a.cap0 * TS : scr0 + (size_t)(s % S::NSCR) * a.cap1 * TS;
      const unsigned char *stage = reinterpret_cast<const unsigned char *>(stage_t);
      unsigned char *obase = gout;
      int64_t orhs = a.out_rhs;
      if (a.entries) {
        const BatchEntry &be = a.entries[w / a.nrhs];
        obase = reinterpret_cast<unsigned char *>(be.out);
        orhs = be.out_rhs;
      }
      unsigned char *rout = obase + (size_t)(w % a.nrhs) * orhs * sizeof(C);
      for (int j = lane; j < n_oruns; j += 32) {
        const Run rn = oruns[j];
        bulk_s2g(rout + (size_t)rn.start * S::tile_bytes, stage + (size_t)rn.slot * S::tile_bytes,
                 (unsigned)(rn.count * S::tile_bytes));
      }
      bulk_commit();
      bulk_wait_read();  // the slot may be refilled after this
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
      // the next item; a counter's latency overlaps the write-back's stores
      long long w = blockIdx.x;
      if (it > 0 && lane == 0) w = (long long)gridDim.x + (long long)atomicAdd(a.sched, 1ull);
      if (wb) {
        write_back(s, slot_w[s]);
        slot_it[s] = -1;
      }
      w = __shfl_sync(0xffffffffu, w, 0);
      if (w >= total) {
        // no more work: the consumers stop at iteration it (the phase completes without
        // data)
        if (lane == 0) {
          *end_it = it;
          mbar_arrive(&full[s]);
        }
        phase_it[s] = it;
        __syncwarp();
        break;
      }
      const long long ch = w / a.nrhs;
      const int r = (int)(w % a.nrhs);
      const ChunkDesc cd = a.entries ? a.entries[ch].d : a.chunks[ch];
      const unsigned char *blob = a.entries ? a.entries[ch].blob : a.blob;
      const Run *runs = a.entries ? a.entries[ch].runs : a.runs;
      const unsigned char *ibase =
          a.entries ? reinterpret_cast<const unsigned char *>(a.entries[ch].in) : gin;
      const int64_t irhs = a.entries ? a.entries[ch].in_rhs : a.in_rhs;
      slot_it[s] = it;
      slot_w[s] = w;
      if (a.inject_stall && it == 0) {
        // test hook: the first chunk never arrives (every later copy still follows the
        // predecessor grid, as in a normal launch)
        if (!waited) {
          pdl_wait();
          waited = true;
        }
        continue;
      }
      unsigned char *meta_s = meta0 + (size_t)s * a.meta_bytes;
      unsigned char *in_s = reinterpret_cast<unsigned char *>(slot0 + (size_t)s * a.cap0 * TS);
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[s], (unsigned)(cd.blob_bytes + cd.n_in * (int)S::tile_bytes));
        bulk_g2s(meta_s, blob + cd.blob_off, (unsigned)cd.blob_bytes, &full[s]);
      }
      __syncwarp();
      if (!waited) {
        // the first chunk's program is in flight; its inputs are the predecessor's outputs
        pdl_wait();
        waited = true;
      }
      const unsigned char *rin = ibase + (size_t)r * irhs * sizeof(C);
      for (int j = lane; j < cd.n_runs; j += 32) {
        const Run rn = runs[cd.run_off + j];
        bulk_g2s(in_s + (size_t)rn.slot * S::tile_bytes, rin + (size_t)rn.start * S::tile_bytes,
                 (unsigned)(rn.count * S::tile_bytes), &full[s]);
      }
      phase_it[s] = it;
    }
    // the outputs of the iteration before the last
    const int sl = (it + 1) & 1;
    if (!failed && slot_it[sl] >= 0) {
      if (wait_staged(sl, slot_it[sl])) write_back(sl, slot_w[sl]);
      else failed = true;
    }
    if (!waited) pdl_wait();
    if (failed && lane == 0) atomicOr(a.status, 1);
    // copies still in flight land before the block exits
    for (int s = 0; s < 2; ++s) {
      const bool ok = phase_it[s] < 0 || mbar_wait(&full[s], (phase_it[s] >> 1) & 1, a.wait_limit);
      if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(a.status, 2);
    }
    bulk_wait_all();  // outputs written before the block exits
    if (lane == 0) {
      // the last block done with the counter resets it for the next launch of this stage
      __threadfence();
      if (atomicAdd(&a.sched[1], 1ull) == (unsigned long long)gridDim.x - 1) {
        atomicExch(&a.sched[0], 0ull);
        atomicExch(&a.sched[1], 0ull);
      }
    }
    return;
  }

  // ---------------- consumer warps (shared memory only, but for the status word)
  pdl_wait();
  for (int it = 0;; ++it) {
    const int s = it & 1, use = it >> 1;
    const bool ok = mbar_wait(&full[s], use & 1, a.wait_limit);
    if (consumer_any(!ok)) {  // every consumer warp leaves together
      if (tid == 0) atomicOr(a.status, 4);
      break;
    }
    if (it == *static_cast<volatile int *>(end_it)) break;  // written before that phase completed
    const unsigned char *meta_s = meta0 + (size_t)s * a.meta_bytes;
    C *in_s = slot0 + (size_t)s * a.cap0 * TS;
    C *scr = scr0 + (size_t)(s % S::NSCR) * a.cap1 * TS;
    const int32_t *hdr = reinterpret_cast<const int32_t *>(meta_s);
    const int NP = hdr[0];
    const Item *ip = reinterpret_cast<const Item *>(meta_s + kBlobHeader);
    // pass j (axis j mod D) reads the buffer pass j-1 wrote and writes the scratch buffer
    // (even j) or the input buffer (odd j); a barrier between passes
    for (int j = 0; j < NP; j += D) {
      if (j > 0) consumer_sync();
      run_pass<R, D, P, 0, ADJ>(ip, hdr[4 + j], hdr[4 + kMaxPasses + j], (j & 1) ? scr : in_s,
                                (j & 1) ? in_s : scr, warp, lane);
      ip += hdr[4 + j];
      consumer_sync();
      run_pass<R, D, P, 1, ADJ>(ip, hdr[5 + j], hdr[5 + kMaxPasses + j], (j & 1) ? in_s : scr,
                                (j & 1) ? scr : in_s, warp, lane);
      ip += hdr[5 + j];
      if constexpr (D == 3) {
        consumer_sync();
        run_pass<R, D, P, (D == 3 ? 2 : 0), ADJ>(ip, hdr[6 + j], hdr[6 + kMaxPasses + j], (j & 1) ? scr : in_s,
                                                 (j & 1) ? in_s : scr, warp, lane);
        ip += hdr[6 + j];
      }
    }
    fence_async_shared();  // the staged tiles are visible to the bulk stores
    consumer_sync();
    if (tid == 0) mbar_arrive(&staged[s]);
  }
}

}  // namespace bfly
