/*
 * bfly.h — C ABI of the GB300 butterfly sparse Fourier transform.
 *
 * The transform (eq. 1.1, Sec. 1):   u_i = sum_j exp(2 pi i x_i . k_j / N) f_j
 * for targets x_i and sources k_j in [0, N]^dim (dim = 2 or 3), computed by the
 * butterfly algorithm of Sec. 2.2 with p^dim equivalent charges per box pair.
 *
 * Conventions shared by every entry point
 *   - Complex arrays are interleaved (re, im) pairs: complex64 (BFLY_C64, two floats) or
 *     complex128 (BFLY_C128, two doubles).  A batch of nrhs right-hand sides is stored
 *     right-hand side major: f[r][j] at f + r*nk, u[r][i] at u + r*nx (in elements).
 *   - Points are row-major doubles, x[i*dim + d], in the caller's order; results come
 *     back in the caller's order.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *     Execution entry points are asynchronous on that stream and never synchronise the
 *     device, except bfly_execute_host (which returns once its result is on the host).
 *   - No entry point throws; every failure returns a status and records a message that
 *     bfly_last_error() returns (thread-local, valid until the next call on the thread).
 *   - A plan may be used by one stream at a time: its workspace is shared by its calls.
 */
#ifndef BFLY_H
#define BFLY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bfly_plan_s *bfly_plan_t;
typedef struct bfly_batch_s *bfly_batch_t;

typedef enum {
  BFLY_OK = 0,
  BFLY_ERR_INVALID_ARG = 1,   /* bad dimension, p, N, point, pointer or size */
  BFLY_ERR_OUT_OF_MEMORY = 2, /* a host or device allocation failed */
  BFLY_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
  BFLY_ERR_UNSUPPORTED = 4,   /* valid request outside what the library implements */
  BFLY_ERR_TIMEOUT = 5        /* a bounded device-side wait gave up */
} bfly_status;

typedef enum { BFLY_C64 = 0, BFLY_C128 = 1 } bfly_dtype;

/* Arithmetic of the butterfly applies.  FP32: complex64 charges, FP32 operators and
 * accumulation, operators and per-point weights built in FP64.  FP64: complex128
 * throughout (the plain FP64 GPU butterfly).  TC (2D): the FP32 plan with the recursive
 * step (Sec. 2.2 step 3) on the tensor cores for many right-hand sides: eight right-hand
 * sides of a box pair form the columns of one real product R(C) X with the operator in
 * real form, as TF32 MMAs compensated to FP32 accuracy (both operands split hi + lo,
 * three products), FP32 accumulation; leaf and final steps as FP32. */
typedef enum { BFLY_PREC_FP64 = 0, BFLY_PREC_FP32 = 1, BFLY_PREC_TC = 2 } bfly_precision;

/* Build only the host plan: no device memory is touched, execution entry points return
 * BFLY_ERR_INVALID_ARG; bfly_plan_info and bfly_plan_stage still work.  */
#define BFLY_FLAG_HOST_ONLY 1u
/* Test hook for failure detection: every launch of the recursive step withholds the data
 * of its first block of work and waits at most about a millisecond for it, so the bounded
 * waits time out and set the device status word (results are then invalid). */
#define BFLY_FLAG_TEST_STALL 2u

/* Autotune the recursive step: build the plan for each candidate configuration, time a
 * forward sweep of each with max_nrhs right-hand sides (median of three after a warm-up),
 * and keep the fastest.  Candidates: the shared-memory budget per block (which sets how
 * many tiles, and so box pairs, one block takes at a time and how many blocks share an
 * SM) x the stages per launch (2D: 3, 2, 1; 3D: one); for an FP32 plan in 2D with
 * max_nrhs >= 4, the right-hand-side grouped step (BFLY_FLAG_RHS_GROUPS) at two budgets
 * and two stage counts; with max_nrhs >= 8 also the tensor-core recursive step
 * (BFLY_PREC_TC) at two budgets and two stage counts; then the best FP32 or FP64
 * candidate with the single-launch sweep (BFLY_FLAG_DATAFLOW) switched the other way (on,
 * in 2D: at two and three stages per step).
 * With tune_cache set, a choice recorded there for the same GPU, dim, p, requested
 * precision, nrhs and size class is reused, and new choices are appended.
 * bfly_plan_info_t reports the chosen precision, budget, stages, whether the right-hand
 * sides are grouped (rhs_groups) and whether the sweep runs in one launch (dataflow). */
#define BFLY_FLAG_AUTOTUNE 4u
/* One stage per launch of the recursive step also in 2D (no stages fused in shared
 * memory): the unfused programs of Sec. 2.2 step 3, for comparison and testing. */
#define BFLY_FLAG_ONE_STAGE 8u
/* FP32 plans in 2D: the recursive step takes the right-hand sides eight at a time (each
 * work item a chunk x eight right-hand sides, tiles right-hand side major in shared
 * memory, a 32-lane step four fibres x eight right-hand sides) with the same paired FP32
 * multiply-adds, in the same order, as the default kernel: the same results, a layout
 * with fewer shared-memory bank conflicts for many right-hand sides.  Default budget
 * 110 KB per block. */
#define BFLY_FLAG_RHS_GROUPS 16u
/* FP32 and FP64 plans: the whole recursive step of a transform (Sec. 2.2 step 3, stages
 * L-1 .. 0) in one launch.  The chunks of all its steps form one list, step after step,
 * and a block starts a chunk of a step as soon as the chunks of the step before it whose
 * outputs it reads have written them (a flag per chunk and right-hand side in device
 * memory, published with release and read with acquire semantics), instead of after the
 * launch of the whole step before it has ended.  Every boundary between two steps has its
 * own charge buffer: the plan holds steps - 1 more stage buffers than without the flag.
 * bfly_execute, bfly_execute_adjoint, bfly_execute_host and bfly_execute_events run the
 * sweep this way (bfly_execute_events then records its events between the recursive
 * step's steps back to back, after the one launch); the split, no-allocation and batch
 * entry points launch step by step as without the flag.  The results are bit-identical
 * to those of the same steps launched one by one (in 2D the flag makes two stages per step
 * the default: a plan without it built with stages = 2).  BFLY_ERR_UNSUPPORTED with BFLY_PREC_TC or
 * BFLY_FLAG_RHS_GROUPS; with BFLY_FLAG_AUTOTUNE, candidates on those steps are built
 * without it. */
#define BFLY_FLAG_DATAFLOW 32u

typedef struct {
  int prec;                /* bfly_precision; default BFLY_PREC_FP32 */
  int max_nrhs;            /* workspace is sized for up to this many right-hand sides (>= 1) */
  unsigned flags;          /* BFLY_FLAG_* */
  int smem_kb;             /* shared memory per block for the recursive step, 0 = default
                              (2D: 72 KB FP32, 55 KB FP64; 3D: 73 KB; BFLY_PREC_TC: 110 KB) */
  const char *tune_cache;  /* autotuning cache file (text), or NULL */
  int stages;              /* at most this many stages per launch of the recursive step:
                              2D 1..3 (0 = default 3, or 2 with BFLY_FLAG_DATAFLOW), 3D 1..2
                              (0 = default 1; larger values are taken as 2);
                              BFLY_FLAG_ONE_STAGE sets 1 */
  int reserved;            /* must be zero */
} bfly_opts;

typedef struct {
  int dim, p, L;                /* L = ceil(log2 N) levels below the root (0 if N <= 1) */
  int prec;                     /* bfly_precision of the plan */
  double N;
  double rho;                   /* N / 2^L, in (1/2, 1]; the points are scaled by 1/sqrt(rho) */
  int64_t nx, nk;               /* number of targets and sources */
  int64_t total_pairs;          /* sum over stages t of nA(L-t) * nK(t) */
  int64_t max_pairs;            /* largest stage */
  int64_t workspace_bytes;      /* device bytes held by the plan */
  int64_t tiles_read_fwd;       /* recursive step: charge tiles read, forward, one RHS */
  int64_t tiles_written_fwd;    /* recursive step: charge tiles written, forward */
  int64_t jobs_fwd;             /* (output box pair, child) pairs of the recursive step */
  int64_t chunks_fwd;           /* blocks of work of the recursive step, all stages */
  double flops_fwd;             /* real flops of the recursive step as executed, one RHS */
  double lane_use_fwd;          /* recursive step: fraction of the issued lanes that work
                                   (operator groups are processed 32 fibres at a time) */
  int smem_kb;                  /* shared-memory budget per block of the recursive step */
  int blocks_per_sm;            /* resident blocks of the recursive step per SM */
  double tuned_ms;              /* autotuning: time of the chosen candidate (0 if not tuned) */
  double plan_seconds;          /* host wall time of bfly_plan_create */
  int steps;                    /* launches of the recursive step per transform: up to three
                                   stages each in 2D, one in 3D (bfly_plan_step) */
  int stages_per_launch;        /* the most stages of one launch the plan was built for */
  int rhs_groups;               /* 1 when built with BFLY_FLAG_RHS_GROUPS */
  int dataflow;                 /* 1 when built with BFLY_FLAG_DATAFLOW */
} bfly_plan_info_t;

/*
 * bfly_plan_create — Sec. 2.2 step 1 and everything that depends only on the points.
 * With L = ceil(log2 N) and s = sqrt(2^L / N) (s = 1 when N is a power of two, the
 * setting of Sec. 2.2), x.k/N = (s x).(s k)/2^L: the plan builds the transform of
 * N' = 2^L on the scaled points, which lie in [0, 2^L]^dim, with unit leaves.  It assigns
 * every scaled point to its leaf (index min(floor(s x), 2^L - 1) per axis), sorts the
 * points by leaf in Morton order, builds the non-empty boxes of every level of T_X and
 * T_K with their child ranges, the transfer operators (eqs. M1 and E1 combined, built in
 * FP64), and the per-point interpolation weights of steps 2 and 4; uploads all of it and
 * allocates two charge buffers of the largest stage (Sec. 2.2: two adjacent levels are
 * live).
 *   out      receives the plan; *out is NULL on failure.
 *   dim      2 or 3.   N: finite, > 0.   p: 3, 5, 7 or 9.
 *   x, k     host arrays [nx][dim] and [nk][dim], every coordinate finite and in [0,N];
 *            copied, the caller keeps ownership.  nx, nk >= 0 (x or k may be NULL when
 *            its count is 0: the transform then returns zeros, or nothing).
 *   opts     NULL for defaults.
 * Errors: INVALID_ARG (any of the above), UNSUPPORTED (even p; N beyond 2^30 in 2D or
 * 2^20 in 3D; BFLY_PREC_TC in 3D; a p or precision whose workspace does not fit on
 * chip), OUT_OF_MEMORY,
 * CUDA.
 * The device current at the call owns the plan's memory; execute on that device.
 */
bfly_status bfly_plan_create(bfly_plan_t *out, int dim, double N, int64_t nx,
                             const double *x, int64_t nk, const double *k, int p,
                             const bfly_opts *opts);

/* Frees the plan and its device memory (after synchronising with nothing: the caller
 * must ensure no execution on the plan is in flight).  NULL is ignored. */
void bfly_plan_destroy(bfly_plan_t plan);

/*
 * bfly_execute — the forward transform, Sec. 2.2 steps 2-4: leaf equivalent charges,
 * the recursive step for t = L-1 .. 0, and evaluation at the targets.
 *   f   device [nrhs][nk] sources (dtype), read only.
 *   u   device [nrhs][nx] potentials (dtype), overwritten.
 *   1 <= nrhs <= max_nrhs of the plan.  f and u must not overlap.  A pointer may be NULL
 *   when its side has no points; with no sources u is set to zero.
 * The arithmetic is the plan's precision whatever the I/O dtype.
 */
bfly_status bfly_execute(bfly_plan_t plan, const void *f, void *u, int nrhs, int dtype,
                         void *stream);

/*
 * bfly_execute_adjoint — the exact conjugate transpose of bfly_execute (the same sweep
 * run backwards, T_X to T_K, with conjugate-transposed operators):
 *   f_j ~= sum_i exp(-2 pi i x_i . k_j / N) u_i.
 *   u   device [nrhs][nx] input;  f  device [nrhs][nk] output, overwritten.
 */
bfly_status bfly_execute_adjoint(bfly_plan_t plan, const void *u, void *f, int nrhs,
                                 int dtype, void *stream);

/*
 * bfly_execute_host — bfly_execute (adjoint = 0) or bfly_execute_adjoint (adjoint = 1)
 * on HOST buffers, returning once the result is in out_host.  When both buffers are
 * pinned (page-locked, e.g. cudaHostAlloc or cudaHostRegister) the leaf step reads the
 * input and the final step writes the result directly in host memory through their
 * device mappings (no staging copies); otherwise the input is copied to the plan's device
 * staging buffer, the sweep runs, and the result is copied back.  in: [nrhs][nk]
 * (forward) or [nrhs][nx] (adjoint).
 */
bfly_status bfly_execute_host(bfly_plan_t plan, const void *in_host, void *out_host,
                              int nrhs, int dtype, int adjoint, void *stream);

/*
 * bfly_direct — eq. 1.1 summed term by term on the GPU (O(nx*nk)), the exact reference
 * and the GPU direct-sum baseline.  The phase x.k/N is formed and reduced mod 1 in FP64;
 * the exponential is evaluated in the plan's precision, sums are FP32 within tiles of
 * sources and FP64 across tiles for an FP32 plan, FP64 throughout for an FP64 plan.
 *   adjoint = 0: in = f [nrhs][nk] -> out = u [nrhs][nx];
 *   adjoint = 1: in = u [nrhs][nx] -> out = f [nrhs][nk] with exp(-2 pi i x.k/N).
 */
bfly_status bfly_direct(bfly_plan_t plan, const void *in, void *out, int nrhs, int dtype,
                        int adjoint, void *stream);

/*
 * bfly_execute_events — bfly_execute (adjoint = 0) or bfly_execute_adjoint (adjoint = 1)
 * that also records caller-owned CUDA events on `stream`: events[i] just before kernel
 * launch i and events[S+2] after the last launch (S = bfly_plan_info_t.steps), so that the
 * elapsed time between events[i] and events[i+1] is the device time of launch i.  Launch
 * order: forward [leaf step, the S recursive-step launches for stages L-1 .. 0 (one or
 * two stages each), final step]; adjoint [final step adjoint, the S launches in reverse,
 * leaf step adjoint].  n_events must be S + 3; NULL entries are skipped.  Asynchronous
 * like bfly_execute: nothing is synchronised or allocated.
 */
bfly_status bfly_execute_events(bfly_plan_t plan, const void *in, void *out, int nrhs,
                                int dtype, int adjoint, void *stream, void *const *events,
                                int n_events);

/*
 * Split sweep, for a transform sharded over ranks (the paper has no counterpart; the
 * sweep is Sec. 2.2 steps 2-4 cut at stage t): the first part runs the leaf step and the
 * recursive step down to stage t, the second from stage t on down to stage 0 and the final
 * step.  Ranks that own subtrees of T_K run the first part on their sources, exchange the
 * stage-t charges, and ranks that own subtrees of T_X run the second part for their
 * targets (paper_0801_1524_gb300/sharded.py).
 *   charges  device [nrhs][nA(L-t) * nB(t)][TS] equivalent charges of stage t in the plan's
 *            precision (complex64 or complex128 interleaved), tile iA * nB + iB in the order
 *            of bfly_plan_boxes, TS = the plan's tile stride (p^dim rounded up to an even
 *            count in FP32, p^dim in FP64), rescaled as the recursive step keeps them
 *            (g^{AB}_m = prod_d e^{2 pi i a_d m_d / (p-1)} f^{AB}_m, a the index of A).
 *   t        a stage at a launch boundary of the plan: L, or the last stage of one of the
 *            launches of bfly_plan_step (plans built with stages = 1 have every stage);
 *            otherwise BFLY_ERR_INVALID_ARG.
 * bfly_execute_to_stage   adjoint = 0: f device [nrhs][nk] (dtype) -> the leaf step and
 *                         the recursive step down to stage t -> charges of stage t;
 *                         adjoint = 1: u device [nrhs][nx] -> the final step's transpose and
 *                         the adjoint sweep from stage 0 up to stage t -> charges of stage t.
 * bfly_execute_from_stage adjoint = 0: charges of stage t -> the rest of the sweep and the
 *                         final step -> u device [nrhs][nx] (dtype);
 *                         adjoint = 1: charges of stage t -> the adjoint sweep up to stage L
 *                         and the leaf step's transpose -> f device [nrhs][nk].
 * to_stage(t) followed by from_stage(t) is bfly_execute (adjoint = 0) or
 * bfly_execute_adjoint (adjoint = 1), for every t at a launch boundary.
 * Asynchronous on `stream`; they copy the stage through the plan's charge buffers.
 */
bfly_status bfly_execute_to_stage(bfly_plan_t plan, const void *in, int t, void *charges, int nrhs, int dtype,
                                  int adjoint, void *stream);
bfly_status bfly_execute_from_stage(bfly_plan_t plan, const void *charges, int t, void *out, int nrhs, int dtype,
                                    int adjoint, void *stream);

/*
 * bfly_execute_noalloc — bfly_execute (forward, device buffers) without any allocation:
 * the two charge buffers of the sweep come from a static device array owned by the
 * library (64 MiB in all, 32 MiB per buffer) instead of the plan's workspace.  The paper
 * has no counterpart.  It serves callers that cannot allocate device memory at the time
 * they run the transform: code whose device memory is owned by an external allocator or
 * a fixed memory budget (a framework's caching allocator, a service with a preset
 * footprint), code that must not call cudaMalloc on its execution path (cudaMalloc may
 * synchronise the device and its latency is unbounded), and many plans that share one
 * fixed workspace.  The plan itself must have been created beforehand.
 *   - Sizes: max_pairs * tile * element bytes * nrhs must fit in 32 MiB, otherwise the call
 *     returns BFLY_ERR_INVALID_ARG and says so; nothing is launched then.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current and caches it: make that first call before any stream
 *     capture.  The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 *     routine).
 *   - Every call shares the array and it keeps the last call's contents (nothing in it
 *     needs clearing): calls that overlap on the GPU (other streams, other threads) race.
 * Arguments, layouts and results are those of bfly_execute.
 */
bfly_status bfly_execute_noalloc(bfly_plan_t plan, const void *f, void *u, int nrhs, int dtype,
                                 void *stream);

/*
 * bfly_device_status — waits for the device, then reads and clears the plan's device
 * status word.  Kernels whose bounded waits gave up set bits in it (1: the copy engine
 * side gave up waiting for a free buffer, 2: copies were still in flight at exit, 4: the
 * compute side gave up waiting for data, 8: a block of a BFLY_FLAG_DATAFLOW sweep gave up
 * waiting for the outputs of other blocks) and return early.  *flags (optional) receives
 * the bits.  Returns BFLY_ERR_TIMEOUT when any bit was set, else BFLY_OK.
 */
bfly_status bfly_device_status(bfly_plan_t plan, int *flags);

/*
 * bfly_stream_status — bfly_device_status ordered on one stream: reads the plan's status
 * word after the work already issued to `stream` (NULL: the legacy default stream) and
 * clears it there, waiting for that stream only (work on other streams keeps running).
 * *flags (optional) receives the bits.  Returns BFLY_ERR_TIMEOUT when any bit was set.
 */
bfly_status bfly_stream_status(bfly_plan_t plan, void *stream, int *flags);

/*
 * bfly_measure_peak — arithmetic throughput of the current device's SMs, the denominator
 * of the roofline fraction of the recursive step (the paper has no counterpart): a
 * register-resident loop of independent multiply-add chains on every SM, timed with CUDA
 * events (best of three launches after a warm-up, on a stream of its own; synchronises
 * that stream).  kind 0: FP64 fma; 1: FP32 fma; 2: paired FP32 fma (fma.rn.f32x2, the
 * form of the FP32 recursive step).  *flops_per_s receives 2 flops per multiply-add;
 * *ms (optional) the time of the best launch.  Allocates nothing.
 */
bfly_status bfly_measure_peak(int kind, double *flops_per_s, double *ms);

/*
 * Batches: many independent transforms (each the operation of bfly_execute, Sec. 2.2)
 * run together.  The paper has no counterpart; a batch groups plans of equal dim, p and
 * precision (different N and point sets), aligned at the final stage, and runs one
 * launch of the recursive step per stage t over the work of every plan's launch that
 * starts at stage t (bfly_plan_step), the chunks of all plans scheduled together.
 *
 * bfly_batch_create — plans: count device plans (the caller keeps ownership and must
 *   keep them alive while the batch exists).  The plans must have been created with the
 *   same shared-memory budget (smem_kb).
 *   Errors: INVALID_ARG (NULL, host-only plans, mixed dim / p / precision / device /
 *   tile capacities), UNSUPPORTED, OUT_OF_MEMORY, CUDA.
 * bfly_batch_execute — f[i] (device, [nrhs][nk_i]) -> u[i] (device, [nrhs][nx_i]) for
 *   every plan i, nrhs <= every plan's max_nrhs, asynchronous on `stream`.  On a
 *   non-default stream the launches are captured into a CUDA graph the first time and
 *   the graph is replayed while f, u, nrhs, dtype and stream are unchanged (other values
 *   capture a new graph); on the default stream the launches are issued directly.  The
 *   batch uses the plans' workspaces: do not execute those plans concurrently.
 * bfly_batch_status — like bfly_device_status for the batch's launches.
 * bfly_batch_destroy — frees the batch (not the plans); NULL is ignored.
 */
bfly_status bfly_batch_create(bfly_batch_t *out, int count, const bfly_plan_t *plans);
bfly_status bfly_batch_execute(bfly_batch_t batch, const void *const *f, void *const *u, int nrhs,
                               int dtype, void *stream);
bfly_status bfly_batch_status(bfly_batch_t batch, int *flags);
void bfly_batch_destroy(bfly_batch_t batch);

/* Sizes and counts of the plan (host data; no device access). */
bfly_status bfly_plan_info(bfly_plan_t plan, bfly_plan_info_t *info);

/*
 * bfly_plan_step — the stages of launch s (0 <= s < steps) of the recursive step in the
 * forward sweep: stages *t, *t - 1, .., *t - *levels + 1 (Sec. 2.2 step 3, one launch for
 * them; the adjoint sweep runs the launches in reverse).  BFLY_ERR_INVALID_ARG for s out
 * of range or a NULL pointer.
 */
bfly_status bfly_plan_step(bfly_plan_t plan, int s, int *t, int *levels);

/*
 * bfly_plan_program — a copy of the compiled chunk program of recursive-step launch s
 * (adjoint = 0: forward, 1: adjoint) for inspection and testing.  what = 0: the chunk
 * descriptors (32 bytes each: blob offset and bytes, first run and run count, input
 * tiles, passes, 2 padding), 1: the metadata blobs (per chunk: a 64-byte header {passes,
 * inputs, output runs, 0, items of passes 0..5, two-source items of passes 0..5}, the
 * items of every pass (8 bytes: source slots 0 and 1 (0xffff: none), destination slot,
 * operators gamma*2 + delta of source 0 in bits 0-1 and of source 1 in bits 2-3), the
 * output runs), 2: the input runs (8 bytes each: first global tile, first slot, count).
 * out = NULL: *bytes receives the size; else min(size, cap) bytes are copied to out and
 * *bytes receives the size.  Works for host-only plans.
 */
bfly_status bfly_plan_program(bfly_plan_t plan, int s, int adjoint, int what, void *out, int64_t cap,
                              int64_t *bytes);

/*
 * bfly_plan_boxes — the non-empty boxes of level lev (0 = root .. L) of T_X (side = 0) or
 * T_K (side = 1) in the plan's order (Sec. 2.2 step 1; Morton order, children of a box
 * consecutive): out[i][d] = integer index of box i along axis d.  A stage-t charge tile
 * of the stage buffers is at iA * nB + iB with A the box of T_X level L - t and B that of
 * T_K level t in this order.  out = NULL: *n receives the box count; else min(n, cap)
 * boxes are copied.  Works for host-only plans.
 */
bfly_status bfly_plan_boxes(bfly_plan_t plan, int side, int lev, int32_t *out, int64_t cap, int64_t *n);

/* Stage t (0..L): number of non-empty T_X boxes at level L-t (nA) and T_K boxes at
 * level t (nB); the stage holds nA*nB equivalent-charge tiles. */
bfly_status bfly_plan_stage(bfly_plan_t plan, int t, int64_t *nA, int64_t *nB);

/* Message of the last failure on this thread ("" if none). */
const char *bfly_last_error(void);

/* Build identification, e.g. "bfly 0.2 sm_103a". */
const char *bfly_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BFLY_H */
