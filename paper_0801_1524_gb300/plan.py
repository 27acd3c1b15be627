"""Python binding of the butterfly: the same entry points as include/bfly.h, marshalling
PyTorch tensors (device memory and streams) into the C ABI.  No arithmetic happens here;
there is no CPU fallback: a missing or unloadable libbfly.so raises."""
from __future__ import annotations

import ctypes

import numpy as np

from . import native

# "fp32g": FP32 with the recursive step on groups of eight right-hand sides
# (BFLY_FLAG_RHS_GROUPS; the same results as "fp32")
PRECISIONS = {"fp64": native.BFLY_PREC_FP64, "fp32": native.BFLY_PREC_FP32, "tc": native.BFLY_PREC_TC,
              "fp32g": native.BFLY_PREC_FP32}


def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.complex64:
        return native.BFLY_C64
    if t.dtype == torch.complex128:
        return native.BFLY_C128
    raise TypeError(f"expected complex64 or complex128, got {t.dtype}")


_raw_stream = None


def _stream_ptr(stream):
    """cudaStream_t of `stream` (a torch.cuda.Stream, a raw handle as int, or None for the
    current stream of the current device)."""
    global _raw_stream
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    torch = _torch()
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream)
    if _raw_stream is None:
        # the current stream's handle without building a Stream object on every call
        fn = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        _raw_stream = (lambda: fn(torch.cuda.current_device())) if fn else \
            (lambda: torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(_raw_stream())


class Plan:
    """Butterfly plan for targets x [nx, dim] and sources k [nk, dim] in [0, N]^dim.

    forward(f):  u_i = sum_j exp(2 pi i x_i.k_j/N) f_j  (Sec. 2.2, approximate to eps(p))
    adjoint(u):  the exact conjugate transpose of forward
    direct(f):   eq. 1.1 summed term by term on the GPU
    """

    def __init__(self, x, k, N: float, p: int, precision: str = "fp32", max_nrhs: int = 1,
                 host_only: bool = False, smem_kb: int = 0, flags: int = 0,
                 autotune: bool = False, tune_cache: str | None = None, stages: int = 0,
                 dataflow: bool = False):
        lib = native.load()
        x = np.ascontiguousarray(x, dtype=np.float64)
        k = np.ascontiguousarray(k, dtype=np.float64)
        if x.ndim != 2 or k.ndim != 2 or x.shape[1] != k.shape[1]:
            raise ValueError("x and k must be [n, dim] arrays with the same dim")
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        self.dim = x.shape[1]
        self.N = float(N)
        self.p = int(p)
        self.nx, self.nk = x.shape[0], k.shape[0]
        self.precision = precision  # requested; info()["prec"] is the one built (autotuning)
        self.max_nrhs = int(max_nrhs)
        opts = native.Opts()
        opts.prec = PRECISIONS[precision]
        opts.max_nrhs = self.max_nrhs
        opts.flags = ((native.BFLY_FLAG_HOST_ONLY if host_only else 0) |
                      (native.BFLY_FLAG_AUTOTUNE if autotune else 0) |
                      (native.BFLY_FLAG_RHS_GROUPS if precision == "fp32g" else 0) |
                      (native.BFLY_FLAG_DATAFLOW if dataflow else 0) | int(flags))
        opts.smem_kb = int(smem_kb)
        opts.stages = int(stages)
        self._tune_cache = tune_cache.encode() if tune_cache else None
        opts.tune_cache = self._tune_cache
        h = ctypes.c_void_p()
        self._lib = lib
        self._h = None
        native.check(lib.bfly_plan_create(ctypes.byref(h), self.dim, self.N, self.nx,
                                          x.ctypes.data, self.nk, k.ctypes.data, self.p,
                                          ctypes.byref(opts)), "bfly_plan_create")
        self._h = h

    # ---- lifetime
    def close(self):
        if self._h is not None:
            self._lib.bfly_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- introspection
    def device_status(self) -> int:
        """Waits for the device, reads and clears the status word (0 = no wait gave up)."""
        flags = ctypes.c_int(0)
        st = self._lib.bfly_device_status(self._h, ctypes.byref(flags))
        if st not in (native.BFLY_OK, 5):
            native.check(st, "bfly_device_status")
        return flags.value

    def stream_status(self, stream=None) -> int:
        """bfly_stream_status: the status word read and cleared in the order of `stream`
        (default: the current stream), waiting for that stream only."""
        flags = ctypes.c_int(0)
        st = self._lib.bfly_stream_status(self._h, _stream_ptr(stream), ctypes.byref(flags))
        if st not in (native.BFLY_OK, 5):
            native.check(st, "bfly_stream_status")
        return flags.value

    def info(self) -> dict:
        inf = native.PlanInfo()
        native.check(self._lib.bfly_plan_info(self._h, ctypes.byref(inf)), "bfly_plan_info")
        return {name: getattr(inf, name) for name, _ in native.PlanInfo._fields_}

    def steps(self) -> list:
        """[(t, levels)] per launch of the recursive step (forward order): stages t .. t-levels+1."""
        out = []
        for s in range(self.info()["steps"]):
            t, lev = ctypes.c_int(), ctypes.c_int()
            native.check(self._lib.bfly_plan_step(self._h, s, ctypes.byref(t), ctypes.byref(lev)),
                         "bfly_plan_step")
            out.append((t.value, lev.value))
        return out

    def program(self, s: int, adjoint: bool = False) -> dict:
        """bfly_plan_program: the chunk program of recursive-step launch s as numpy arrays
        {"chunks": int32 [n][8], "blob": uint8 [bytes], "runs": uint8 [n_runs * 8]}."""
        out = {}
        for what, name in ((0, "chunks"), (1, "blob"), (2, "runs")):
            n = ctypes.c_int64()
            native.check(self._lib.bfly_plan_program(self._h, s, int(adjoint), what, None, 0, ctypes.byref(n)),
                         "bfly_plan_program")
            buf = np.zeros(n.value, dtype=np.uint8)
            native.check(self._lib.bfly_plan_program(self._h, s, int(adjoint), what, buf.ctypes.data, n.value,
                                                     ctypes.byref(n)), "bfly_plan_program")
            out[name] = buf
        out["chunks"] = out["chunks"].view(np.int32).reshape(-1, 8)
        return out

    def boxes(self, side: str, lev: int) -> np.ndarray:
        """bfly_plan_boxes: int32 [n][dim] box indices of level `lev` of T_X (side "x") or
        T_K (side "k") in the plan's (Morton) order."""
        sd = {"x": 0, "k": 1}[side]
        n = ctypes.c_int64()
        native.check(self._lib.bfly_plan_boxes(self._h, sd, lev, None, 0, ctypes.byref(n)), "bfly_plan_boxes")
        out = np.zeros((n.value, self.dim), dtype=np.int32)
        native.check(self._lib.bfly_plan_boxes(self._h, sd, lev, out.ctypes.data, n.value, ctypes.byref(n)),
                     "bfly_plan_boxes")
        return out

    def stages(self) -> list:
        """[(t, nA, nB)] for t = 0..L: stage t pairs nA T_X boxes with nB T_K boxes."""
        out = []
        L = self.info()["L"]
        for t in range(L + 1):
            a, b = ctypes.c_int64(), ctypes.c_int64()
            native.check(self._lib.bfly_plan_stage(self._h, t, ctypes.byref(a), ctypes.byref(b)),
                         "bfly_plan_stage")
            out.append((t, a.value, b.value))
        return out

    # ---- execution on device tensors
    def _prep(self, t, n, name):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        squeeze = t.dim() == 1
        t2 = t.reshape(1, t.shape[0]) if squeeze else t
        if t2.dim() != 2 or t2.shape[1] != n:
            raise ValueError(f"{name} must be [{n}] or [nrhs, {n}]")
        return t2.contiguous(), squeeze

    def _run(self, fn, src, n_in, n_out, out, stream, name):
        torch = _torch()
        s, squeeze = self._prep(src, n_in, name)
        if out is None:
            out = torch.empty((s.shape[0], n_out), dtype=s.dtype, device=s.device)
        o2 = out.reshape(s.shape[0], n_out)
        if o2.dtype != s.dtype or not o2.is_contiguous():
            raise ValueError("out must be contiguous with the input's dtype")
        native.check(fn(self._h, ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(o2.data_ptr()),
                        s.shape[0], _dtype_code(s), _stream_ptr(stream)), name)
        return out.reshape(-1) if squeeze and out is not None and out.dim() == 2 else out

    def forward(self, f, out=None, stream=None):
        return self._run(self._lib.bfly_execute, f, self.nk, self.nx, out, stream, "bfly_execute")

    def forward_noalloc(self, f, out=None, stream=None):
        """bfly_execute_noalloc: the forward transform with the library's static workspace,
        for callers that cannot allocate device memory when they run it (an external
        allocator or fixed memory budget owns the device memory, or cudaMalloc's device
        synchronisation is not acceptable on their execution path)."""
        return self._run(self._lib.bfly_execute_noalloc, f, self.nk, self.nx, out, stream,
                         "bfly_execute_noalloc")

    def _charge_dtype(self):
        torch = _torch()
        return torch.complex128 if self.precision == "fp64" or self.info()["prec"] == native.BFLY_PREC_FP64 \
            else torch.complex64

    def boundaries(self) -> list:
        """Stages at the launch boundaries of the sweep (where it can be split): L and the
        last stage of every recursive-step launch."""
        return [self.info()["L"]] + [t - lev + 1 for t, lev in self.steps()]

    def to_stage(self, v, t: int, out=None, adjoint: bool = False, stream=None):
        """bfly_execute_to_stage: forward, the leaf step and the recursive step down to stage
        t of sources v [nrhs, nk]; adjoint, the final step's transpose and the adjoint sweep
        up to stage t of potentials v [nrhs, nx].  Returns the stage-t charges
        [nrhs, nA * nB * TS] (plan precision, plan tile order)."""
        torch = _torch()
        s, _ = self._prep(v, self.nx if adjoint else self.nk, "v")
        nA, nB = self.stages()[t][1:]
        pd = self.p ** self.dim
        ts = pd if self._charge_dtype() == torch.complex128 else pd + (pd & 1)
        if out is None:
            out = torch.empty((s.shape[0], nA * nB * ts), dtype=self._charge_dtype(), device=s.device)
        if out.dtype != self._charge_dtype() or not out.is_contiguous() or out.numel() != s.shape[0] * nA * nB * ts:
            raise ValueError("charges must be contiguous [nrhs, nA * nB * TS] of the plan's precision")
        native.check(self._lib.bfly_execute_to_stage(self._h, ctypes.c_void_p(s.data_ptr()), int(t),
                                                     ctypes.c_void_p(out.data_ptr()), s.shape[0],
                                                     _dtype_code(s), int(adjoint), _stream_ptr(stream)),
                     "bfly_execute_to_stage")
        return out

    def from_stage(self, charges, t: int, out=None, dtype=None, adjoint: bool = False, stream=None):
        """bfly_execute_from_stage: stage-t charges -> forward, potentials [nrhs, nx];
        adjoint, sources [nrhs, nk] (dtype: the charges' complex type unless given)."""
        torch = _torch()
        c = charges.contiguous()
        if c.dtype != self._charge_dtype():
            raise ValueError("charges must have the plan's precision")
        nrhs = c.shape[0]
        if out is None:
            out = torch.empty((nrhs, self.nk if adjoint else self.nx), dtype=dtype or c.dtype, device=c.device)
        native.check(self._lib.bfly_execute_from_stage(self._h, ctypes.c_void_p(c.data_ptr()), int(t),
                                                       ctypes.c_void_p(out.data_ptr()), nrhs, _dtype_code(out),
                                                       int(adjoint), _stream_ptr(stream)), "bfly_execute_from_stage")
        return out

    def adjoint(self, u, out=None, stream=None):
        return self._run(self._lib.bfly_execute_adjoint, u, self.nx, self.nk, out, stream,
                         "bfly_execute_adjoint")

    def direct(self, v, adjoint: bool = False, out=None, stream=None):
        fn = lambda h, a, b, n, dt, st: self._lib.bfly_direct(h, a, b, n, dt, int(adjoint), st)
        n_in, n_out = (self.nx, self.nk) if adjoint else (self.nk, self.nx)
        return self._run(fn, v, n_in, n_out, out, stream, "bfly_direct")

    def with_events(self, v, events, adjoint: bool = False, out=None, stream=None):
        """bfly_execute_events: records the torch.cuda.Event list `events` (info()["steps"]
        + 3 of them, already recorded once so that they exist) around every kernel launch."""
        arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
        fn = lambda h, a, b, n, dt, st: self._lib.bfly_execute_events(h, a, b, n, dt, int(adjoint),
                                                                      st, arr, len(events))
        n_in, n_out = (self.nx, self.nk) if adjoint else (self.nk, self.nx)
        return self._run(fn, v, n_in, n_out, out, stream, "bfly_execute_events")

    # ---- execution on host buffers (copies inside the call)
    def execute_host(self, v: np.ndarray, adjoint: bool = False, out: np.ndarray | None = None,
                     stream=None) -> np.ndarray:
        v = np.asarray(v)
        one = v.ndim == 1
        v2 = v.reshape(1, -1) if one else v
        if not v2.flags.c_contiguous:
            v2 = np.ascontiguousarray(v2)
        n_in, n_out = (self.nx, self.nk) if adjoint else (self.nk, self.nx)
        dt = v2.dtype
        if v2.shape[1] != n_in or (dt != np.complex64 and dt != np.complex128):
            raise ValueError(f"input must be complex64/complex128 [nrhs, {n_in}]")
        if out is None:
            out = np.empty((v2.shape[0], n_out), dtype=dt)
        elif out.dtype != dt or out.size != v2.shape[0] * n_out or not out.flags.c_contiguous:
            raise ValueError("out must be contiguous [nrhs, n] of the input's dtype")
        st = self._lib.bfly_execute_host(self._h, v2.__array_interface__["data"][0],
                                         out.__array_interface__["data"][0], v2.shape[0],
                                         native.BFLY_C128 if dt == np.complex128 else native.BFLY_C64,
                                         int(adjoint), _stream_ptr(stream))
        if st != native.BFLY_OK:
            native.check(st, "bfly_execute_host")
        return out.reshape(-1) if one and out.ndim == 2 else out


class Batch:
    """Many plans (same dim, p, precision) executed together: one launch of the recursive
    step per starting stage over all of them, captured in a CUDA graph on a non-default
    stream."""

    def __init__(self, plans):
        self._lib = native.load()
        self.plans = list(plans)  # kept alive with the batch
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h for p in self.plans])
        h = ctypes.c_void_p()
        self._h = None
        native.check(self._lib.bfly_batch_create(ctypes.byref(h), len(self.plans), arr),
                     "bfly_batch_create")
        self._h = h

    def close(self):
        if self._h is not None:
            self._lib.bfly_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, fs, us=None, stream=None):
        """fs: list of [nrhs, nk_i] CUDA tensors (same dtype); returns / fills us."""
        torch = _torch()
        fs = [(f if f.dim() == 2 else f.reshape(1, f.shape[0])).contiguous() for f in fs]
        for f, p in zip(fs, self.plans):
            if f.shape[1] != p.nk:
                raise ValueError(f"batch input must be [nrhs, {p.nk}]")
        nrhs = fs[0].shape[0]
        if us is None:
            us = [torch.empty((nrhs, p.nx), dtype=fs[0].dtype, device=fs[0].device) for p in self.plans]
        fa = (ctypes.c_void_p * len(fs))(*[f.data_ptr() for f in fs])
        ua = (ctypes.c_void_p * len(us))(*[u.data_ptr() for u in us])
        native.check(self._lib.bfly_batch_execute(self._h, fa, ua, nrhs, _dtype_code(fs[0]),
                                                  _stream_ptr(stream)), "bfly_batch_execute")
        self._keep = (fs, us)  # the device buffers must outlive the asynchronous launches
        return us

    def device_status(self) -> int:
        flags = ctypes.c_int(0)
        st = self._lib.bfly_batch_status(self._h, ctypes.byref(flags))
        if st not in (native.BFLY_OK, 5):
            native.check(st, "bfly_batch_status")
        return flags.value


def measure_peak(kind: str) -> float:
    """bfly_measure_peak on the current device: flop/s of "fp64" (fma), "fp32" (fma) or
    "fp32x2" (paired fma.rn.f32x2) multiply-add loops on every SM."""
    code = {"fp64": 0, "fp32": 1, "fp32x2": 2}[kind]
    lib = native.load()
    v, ms = ctypes.c_double(), ctypes.c_double()
    native.check(lib.bfly_measure_peak(code, ctypes.byref(v), ctypes.byref(ms)), "bfly_measure_peak")
    return v.value


def butterfly_fn():
    """torch.autograd.Function u = B f with du/df handled by the adjoint sweep."""
    torch = _torch()

    class ButterflyFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, f, plan):
            ctx.plan = plan
            return plan.forward(f)

        @staticmethod
        def backward(ctx, g):
            # PyTorch's complex gradient of a real loss is conj-Wirtinger: for u = B f
            # the gradient with respect to f is B^H g, the adjoint sweep.
            return ctx.plan.adjoint(g.contiguous()), None

    return ButterflyFn


def butterfly(f, plan):
    """Differentiable forward transform: ButterflyFn.apply(f, plan)."""
    return butterfly_fn().apply(f, plan)
