#!/usr/bin/env python3
"""Benchmark of the butterfly sparse Fourier transform on one GB300.

Workload (one "step" = one whole transform: leaf step, the L recursive stages in launches
of up to three stages, final step): 2D, N = 8192, X = circle of radius 0.4 (82,355 targets), K = ellipse 0.45 x 0.3
with a 0.03 sin(5 theta) radial perturbation (80,962 sources), p = 7, one right-hand side
of complex64 Gaussian sources, FP32 arithmetic with FP64-built operators.

Printed: one JSON line with transforms/s (device time, inputs resident), the same through
the host-buffer C-ABI call (e2e), the roofline of the recursive-step kernel, the plain
FP64 GPU butterfly and GPU direct sums on the same plan, and the oracle's CPU direct sum
timed on the host cores.  `--impl reference` times the oracle alone.
Under torchrun with N > 1 every rank runs an independent replica (the single transform
is not sharded); value = transforms of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "transforms/sec and effective |I|*|J|/time vs plain FP64 GPU butterfly at rel L2 err<=1e-6"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["bfly", "reference"], default="bfly")
    ap.add_argument("--workload", default="curve8192")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target wall time of the oracle CPU baseline sample")
    ap.add_argument("--no-baselines", action="store_true")
    ap.add_argument("--nrhs", type=int, default=None,
                    help="right-hand sides (default: 1; star_batch: 16)")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--smem-kb", type=int, default=0,
                    help="shared memory per block of the recursive step (0 = the library default)")
    ap.add_argument("--precision", default="fp32",
                    help="precision of the timed path (fp32, tc); star_batch: comma-separated "
                         "precisions of the batch, the first is the value")
    ap.add_argument("--dataflow", choices=["auto", "on", "off"], default="auto",
                    help="recursive step in one launch (BFLY_FLAG_DATAFLOW); auto: on for FP32 "
                         "plans in 2D, where it is measured faster, off in 3D and for the "
                         "tensor-core step")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and p = 9 companion measurements of the default run")
    return ap.parse_args()


def alu_peaks():
    """Arithmetic peaks of this GPU measured in this run (bfly_measure_peak: register-
    resident multiply-add loops on every SM, CUDA events): TFLOP/s of FP32 fma, paired
    FP32 fma (f32x2, the form the FP32 recursive step issues) and FP64 fma."""
    from paper_0801_1524_gb300.plan import measure_peak
    return {k: measure_peak(k) / 1e12 for k in ("fp32x2", "fp32", "fp64")}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def flush_l2(buf):
    """Evicts L2 between timed steps: a write of a buffer twice the L2 size, then a read of
    it, so that the timed kernels find their inputs in HBM and no dirty line of the flush
    is written back inside the timed region."""
    buf.zero_()
    buf.sum()


def workload(name):
    from paper_0801_1524_gb300 import workloads as w
    return w.WORKLOADS[name]()


def describe(inst, nrhs=1):
    return {"workload": f"{inst.name}: {inst.dim}D, N={int(inst.N)}, p={inst.p}, "
                        f"{inst.x.shape[0]} targets, {inst.k.shape[0]} sources, {nrhs} RHS, "
                        "complex64 Gaussian sources (seed 0)",
            "N": int(inst.N), "p": inst.p, "dim": inst.dim, "nx": int(inst.x.shape[0]),
            "nk": int(inst.k.shape[0]), "nrhs": nrhs,
            "l2": "flushed between steps (256 MB written, then read back so that no dirty line "
                  "is left for the timed kernels to write back); per-step CUDA events"}


# ---------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.t_on = self.t_off = None

    def mark(self, on: bool):
        if on:
            self.t_on = time.time()
        else:
            self.t_off = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        loaded = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------- oracle
def oracle_direct_rate(inst, f, seconds: float, seed: int = 12345):
    """The oracle's FP64 direct sum (eq. 1.1) on a seeded subset S of the targets, sized
    to about `seconds` of host time; returns (transforms/s extrapolated, |S|, threads, s)."""
    from oracle.direct import direct, threads
    rng = np.random.default_rng(seed)
    nx = inst.x.shape[0]
    order = rng.permutation(nx)
    probe = order[:min(nx, 256)]
    t0 = time.perf_counter()
    direct(inst.x[probe], inst.k, f, inst.N)
    per_target = (time.perf_counter() - t0) / len(probe)
    m = int(min(nx, max(256, seconds / max(per_target, 1e-9))))
    S = order[:m]
    t0 = time.perf_counter()
    direct(inst.x[S], inst.k, f, inst.N)
    dt = time.perf_counter() - t0
    return (m / nx) / dt, m, threads(), dt


# ---------------------------------------------------------------------------- ranks
def max_over_ranks(ms, dist, device=None):
    """The largest of every rank's step time, on every rank (the job's time: replicas
    run independently, the slowest one bounds the whole job)."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, ms):
    """Transforms per second of the whole job: one transform per rank per step."""
    return world * 1e3 / ms


# ---------------------------------------------------------------------------- main arm
def main_bfly(args, rank, world, dist):
    import torch
    from paper_0801_1524_gb300.plan import Plan

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    inst = workload(args.workload)
    nx, nk = inst.x.shape[0], inst.k.shape[0]
    nrhs = args.nrhs or 1
    prec = args.precision.split(",")[0]
    shp = lambda n: (n,) if nrhs == 1 else (nrhs, n)
    f_np = inst.sources(dtype=np.complex64, nrhs=nrhs).reshape(shp(nk))
    stream = torch.cuda.current_stream()
    f = torch.as_tensor(f_np, device=dev)
    flow = args.dataflow == "on" or (args.dataflow == "auto" and inst.dim == 2 and prec == "fp32")
    plan = Plan(inst.x, inst.k, inst.N, inst.p, precision=prec, smem_kb=args.smem_kb, max_nrhs=nrhs,
                dataflow=flow)
    info = plan.info()
    L = info["L"]
    S = info["steps"]    # steps of the recursive step per transform (bfly_execute_events' marks)
    SL = 1 if info["dataflow"] else S   # its launches
    u = torch.empty(shp(nx), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    alu = alu_peaks()

    def new_events():
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(S + 3)]
        for e in evs:
            e.record(stream)
        return evs

    # warm-up
    for _ in range(max(args.warmup, 3)):
        flush_l2(flush)
        plan.forward(f, out=u)
    torch.cuda.synchronize()

    # one event pair per step around the call a user makes (plan.forward): consecutive
    # launches of a transform may overlap their ramps (programmatic dependent launch)
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    events = [new_events() for _ in range(args.steps)]
    torch.cuda.synchronize()
    vis = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    gpu_index = int(vis[local]) if local < len(vis) and vis[local].strip().isdigit() else local
    clocks = Clocks(gpu_index) if rank == 0 else None
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.mark(True)
    for k in range(args.steps):
        flush_l2(flush)
        step_ev[k][0].record(stream)
        plan.forward(f, out=u)
        step_ev[k][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.mark(False)
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    # per-kernel durations: the same steps again with an event between consecutive
    # launches (which serialises them: each launch's full duration, ramps included)
    for k in range(args.steps):
        flush_l2(flush)
        plan.with_events(f, events[k], out=u)
    torch.cuda.synchronize()
    level_ms = [ev[1].elapsed_time(ev[S + 1]) for ev in events]
    kern_ms = np.array([[ev[i].elapsed_time(ev[i + 1]) for i in range(S + 2)] for ev in events])
    ms = max_over_ranks(float(np.mean(step_ms)), dist, dev)
    clk = clocks.stop() if clocks else None

    # ---- end to end through the host-buffer C-ABI call (copies inside the timed call)
    f_pin = torch.empty(shp(nk), dtype=torch.complex64).pin_memory()
    f_pin.copy_(torch.as_tensor(f_np))
    u_pin = torch.empty(shp(nx), dtype=torch.complex64).pin_memory()
    f_host = f_pin.numpy()
    u_host = u_pin.numpy()
    raw = stream.cuda_stream
    u_out = u_host.reshape(nrhs, -1)
    for _ in range(3):
        plan.execute_host(f_host, out=u_out, stream=raw)
    e2e = []
    for _ in range(max(10, min(args.steps, 100))):
        flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.execute_host(f_host, out=u_out, stream=raw)
        e2e.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e))

    # ---- the adjoint sweep (the gradient's transform) on the same plan, device buffers
    v_adj = torch.empty(shp(nk), dtype=torch.complex64, device=dev)
    for _ in range(3):
        plan.adjoint(u, out=v_adj)
    adj_ms = []
    for _ in range(max(10, min(args.steps, 100))):
        flush_l2(flush)
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_ev.record(stream)
        plan.adjoint(u, out=v_adj)
        b_ev.record(stream)
        b_ev.synchronize()
        adj_ms.append(a_ev.elapsed_time(b_ev))

    if rank != 0:
        return None

    # ---- accuracy of this run and baselines on the same GPU
    out = {}
    u32 = u.to(torch.complex128)
    if not args.no_baselines:
        plan64 = Plan(inst.x, inst.k, inst.N, inst.p, precision="fp64", max_nrhs=nrhs)
        f64 = f.to(torch.complex128)
        u64 = torch.empty(shp(nx), dtype=torch.complex128, device=dev)
        for _ in range(3):
            plan64.forward(f64, out=u64)
        torch.cuda.synchronize()
        ev64 = []
        for _ in range(min(args.steps, 20)):
            flush_l2(flush)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan64.forward(f64, out=u64)
            b.record(stream)
            ev64.append((a, b))
        torch.cuda.synchronize()
        ms64 = float(np.mean([a.elapsed_time(b) for a, b in ev64]))
        rel_vs_fp64 = (torch.linalg.norm(u32 - u64) / torch.linalg.norm(u64)).item()
        # direct sums on the GPU (eq. 1.1), FP64 phase reduction
        ud = torch.empty(shp(nx), dtype=torch.complex128, device=dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan64.direct(f64, out=ud)
        b.record(stream)
        torch.cuda.synchronize()
        ms_direct64 = a.elapsed_time(b)
        ud32 = torch.empty(shp(nx), dtype=torch.complex64, device=dev)
        a.record(stream)
        plan.direct(f, out=ud32)
        b.record(stream)
        torch.cuda.synchronize()
        ms_direct32 = a.elapsed_time(b)
        eps_a = (torch.linalg.norm(u64 - ud) / torch.linalg.norm(ud)).item()
        eps_a32 = (torch.linalg.norm(u32 - ud) / torch.linalg.norm(ud)).item()
        out["baselines"] = {
            "fp64_gpu_butterfly": {"ms": ms64, "transforms_per_s": 1e3 / ms64,
                                   "speedup_of_fp32_path": ms64 / ms},
            "gpu_direct_fp64": {"ms": ms_direct64, "transforms_per_s": 1e3 / ms_direct64},
            "gpu_direct_fp32": {"ms": ms_direct32, "transforms_per_s": 1e3 / ms_direct32},
        }
        out["accuracy"] = {"rel_l2_fp32_vs_fp64_butterfly": rel_vs_fp64,
                           "gate_1e-6_met": rel_vs_fp64 <= 1e-6,
                           "eps_a_fp64_vs_gpu_direct_fp64": eps_a,
                           "eps_a_fp32_vs_gpu_direct_fp64": eps_a32}
        del plan64

    # ---- roofline of the recursive step (the dominant kernel: SL launches per step)
    d, p = inst.dim, inst.p
    PD = p ** d
    # algorithmic units of the recursive step, all stages, one RHS: per (pair, child)
    # 2p^3 complex multiply-adds in 2D (3p^4 in 3D), 8 real flops each; the tiles of the
    # stages between launches read once and written once (p^d complex64 each; the stage
    # inside a two-stage launch stays in shared memory)
    flops = info["jobs_fwd"] * (2 * p ** 3 if d == 2 else 3 * p ** 4) * 8.0 * nrhs
    flops_exec = info["flops_fwd"] * nrhs    # as executed (sum factorisation shares work)
    steps = plan.steps()
    pairs = {t: a * b for t, a, b in plan.stages()}
    bytes_ = sum(pairs[t + 1] + pairs[t - lev + 1] for t, lev in steps) * PD * 8.0 * nrhs
    level_s = float(np.mean(level_ms)) * 1e-3
    per_launch_s = level_s / SL
    hbm_peak, hbm_src = peaks()
    alu_peak = alu["fp32x2"]   # TFLOP/s, measured in this run
    a_alu = flops / SL / per_launch_s / 1e12
    a_exec = flops_exec / SL / per_launch_s / 1e12
    a_hbm = bytes_ / SL / per_launch_s / 1e9
    roof_alu = {"bound": "alu", "achieved": a_alu, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": a_alu / alu_peak, "traffic": None,
                "achieved_executed": a_exec, "frac_executed": a_exec / alu_peak,
                "peak_source": "measured in this run (of measured): paired FP32 fma (f32x2) loop "
                               "on every SM, bfly_measure_peak",
                "frac_note": "frac counts the algorithmic flops (2p^3 complex MACs per pair and "
                             "child); frac_executed the flops the kernel executes (sum "
                             "factorisation, unit columns)"}
    roof_hbm = {"bound": "hbm", "achieved": a_hbm, "peak": hbm_peak, "unit": "GB/s",
                "frac": a_hbm / hbm_peak, "traffic": None,
                "peak_source": f"{hbm_src} copy bandwidth"}
    traffic = level_traffic(dataflow=bool(info["dataflow"]), steps=steps)
    main, alt = (roof_alu, roof_hbm) if roof_alu["frac"] >= roof_hbm["frac"] else (roof_hbm, roof_alu)
    main["traffic"] = traffic
    alt["traffic"] = traffic
    main["kernel"] = (("level_tc_kernel<" if prec == "tc" else "level_kernel<float,") + f"{d},{p}> "
                      + (f"(recursive step in one launch: {S} steps of " if info["dataflow"] else
                         f"(recursive step, {S} launches of ")
                      + "/".join(str(lev) for _, lev in steps) + " stages)")
    main["algorithmic_per_launch"] = {"flops": flops / SL, "bytes": bytes_ / SL,
                                      "executed_flops": flops_exec / SL}
    main["duration"] = ("mean per-launch CUDA-event time of the recursive step, from a second pass "
                        "of the same steps with an event between consecutive launches")
    alt["kernel"] = main["kernel"]
    out["roofline_alt"] = alt
    kern_names = (["leaf"] + [f"level_t{t}" + (f"-{t - lev + 1}" if lev > 1 else "") for t, lev in steps]
                  + ["final"])
    km = kern_ms.mean(axis=0)
    if info["dataflow"]:   # one launch: the marks between its steps are back to back
        out["kernel_ms"] = {"leaf": float(km[0]), f"level_t{L - 1}-0": float(km[1:S + 1].sum()),
                            "final": float(km[S + 1])}
    else:
        out["kernel_ms"] = {n: float(v) for n, v in zip(kern_names, km)}

    value = replica_value(world, ms) * nrhs   # right-hand sides transformed per second
    line = {
        "metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**describe(inst, nrhs), "parallelism": f"replicas{world}" if world > 1 else "single GPU",
                   "precision": "FP32 applies, FP64-built operators and weights" if prec == "fp32" else
                   "recursive step on the tensor cores (TF32 operands split hi + lo, FP32 accumulation), "
                   "FP32 leaf and final steps",
                   "recursive_step": (f"one launch for its {S} steps (BFLY_FLAG_DATAFLOW)" if info["dataflow"]
                                      else f"{S} launches")},
        "ms_stats": {"mean": float(np.mean(step_ms)), "median": float(np.median(step_ms)),
                     "min": float(np.min(step_ms)), "max": float(np.max(step_ms)), "rank": rank},
        "effective_IJ_per_s": value * nx * nk,
        "e2e": {"value": world * nrhs / e2e_s, "unit": "transforms/s", "h2d_bytes_per_step": nk * 8 * nrhs,
                "d2h_bytes_per_step": nx * 8 * nrhs, "ms": e2e_s * 1e3,
                "call": "bfly_execute_host on pinned host buffers (read and written in place "
                        "by the leaf and final steps; H2D and D2H traffic inside the timed call)"},
        "roofline": main,
        "adjoint": {"ms": float(np.mean(adj_ms)), "transforms_per_s": 1e3 / float(np.mean(adj_ms)),
                    "call": "bfly_execute_adjoint (device buffers; the sweep behind the gradient)"},
        "gpu_launches": args.steps * (SL + 2),
        "clocks": clk,
        "plan": {"seconds": info["plan_seconds"], "L": L, "total_pairs": info["total_pairs"],
                 "max_pairs": info["max_pairs"], "workspace_bytes": info["workspace_bytes"]},
    }
    line["alu_peaks_tflops"] = {**alu, "source": "bfly_measure_peak, measured in this run before the "
                                              "timed region"}
    if "baselines" in out:
        # the FP64 butterfly against the measured FP64 fma rate
        fl64 = flops / (out["baselines"]["fp64_gpu_butterfly"]["ms"] * 1e-3) / 1e12
        out["baselines"]["fp64_gpu_butterfly"]["recursive_alg_tflops_over_transform"] = fl64
        out["baselines"]["fp64_gpu_butterfly"]["frac_of_fp64_peak"] = fl64 / alu["fp64"]
    line.update(out)
    if not args.no_extras and world == 1:
        del u
        torch.cuda.empty_cache()
        for key, fn in (("star_batch", lambda: batch_summary(args, dev, flush)), ("p9_rows", lambda: p9_rows(dev))):
            try:
                line[key] = fn()
            except Exception as exc:  # recorded in the line; the headline stands
                line[key] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.no_baselines:
        f_one = f_np if nrhs == 1 else f_np[0]
        rate, m, thr, dt = oracle_direct_rate(inst, f_one.astype(np.complex128), args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": "transforms/s", "cores": thr, "kind": "oracle",
                                "sample": (f"FP64 direct sum (eq. 1.1) over all {nx} targets and all {nk} "
                                           f"sources, {dt:.1f} s (measured)" if m == nx else
                                           f"FP64 direct sum (eq. 1.1) over {m} of {nx} targets "
                                           f"(seeded), all {nk} sources, {dt:.1f} s, extrapolated x nx/|S|")}
    return line


def level_code_hash():
    """sha256 (16 hex digits) of the recursive step's kernel source without its comments and
    blank lines: the key of the committed DRAM-traffic summary."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_0801_1524_gb300", "csrc", "level.cuh")).read()
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in src.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln.strip()).encode()).hexdigest()[:16]


def level_traffic(dataflow, steps):
    """DRAM bytes per recursive-step launch (the one launch of the sweep with dataflow) from
    the committed ncu summary, if it was taken on the current kernel source and the same
    steps; else None."""
    path = os.path.join(ROOT, "profiles", "level_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        if d.get("level_cuh_code_sha256_16") != level_code_hash() or bool(d.get("dataflow", False)) != dataflow:
            return None
        if [list(x) for x in d.get("steps", [])] != [list(x) for x in steps]:
            return None
        return float(d["dram_bytes_per_launch"])
    except Exception:
        return None


# ---------------------------------------------------------------------------- reference arm
def main_reference(args, rank):
    """The oracle's FP64 direct sum (eq. 1.1) on the host cores.  Every timed step
    evaluates the whole target set (so that ms_per_step is measured, not extrapolated)
    when steps x the estimated full-set time fits in 10 minutes; otherwise each step takes
    the largest seeded target sample that does, extrapolated to all targets and labelled
    so.  Warm-up steps use a 256-target sample."""
    if rank != 0:
        return None
    from oracle.direct import direct, threads
    inst = workload(args.workload)
    f = inst.sources(dtype=np.complex128)[0]
    nx = inst.x.shape[0]
    order = np.random.default_rng(12345).permutation(nx)
    probe = order[:min(nx, 256)]
    for _ in range(max(args.warmup, 1)):
        t0 = time.perf_counter()
        direct(inst.x[probe], inst.k, f, inst.N)
        per_target = (time.perf_counter() - t0) / len(probe)
    budget = 600.0 / max(1, args.steps)
    m = nx if per_target * nx <= budget else max(256, int(budget / per_target))
    S = order[:m] if m < nx else np.arange(nx)
    times = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        direct(inst.x[S], inst.k, f, inst.N)
        times.append(time.perf_counter() - t0)
    wall = time.perf_counter() - t_all
    step_s = float(np.mean(times)) * (nx / m)
    value = 1.0 / step_s
    if m == nx:
        sample = (f"FP64 direct sum (eq. 1.1) over all {nx} targets and all {inst.k.shape[0]} "
                  "sources per step (measured, not extrapolated)")
    else:
        sample = (f"FP64 direct sum (eq. 1.1) over {m} of {nx} seeded targets per step, all "
                  f"{inst.k.shape[0]} sources, extrapolated x nx/|S|")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "transforms/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": describe(inst),
            "cpu_baseline": {"value": value, "unit": "transforms/s", "cores": threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": wall, "targets_per_step": m}


def run_batch(insts, nrhs, steps32, steps64, warmup, dev, flush, smem_kb=0, precisions=("fp32",), stages=0):
    """The batched sweep of `insts` (nrhs complex64 right-hand sides each; one recursive-step
    launch per starting stage over all instances, graph replay on a side stream) in each of
    `precisions` ("fp32": paired FP32 multiply-adds; "tc": tensor cores) and in FP64; CUDA
    events around every replay, L2 flushed between replays.  Returns, per precision, the
    time per batch and its accuracy against the FP64 batch."""
    import torch
    from paper_0801_1524_gb300.plan import Batch, Plan
    out = {}
    runs = [(pr, torch.complex64, steps32) for pr in precisions] + [("fp64", torch.complex128, steps64)]
    for prec, dtype, steps in runs:
        plans = [Plan(I.x, I.k, I.N, I.p, precision=prec, max_nrhs=nrhs,
                      smem_kb=smem_kb if prec == precisions[0] else 0,
                      stages=stages if prec == precisions[0] else 0)
                 for I in insts]
        batch = Batch(plans)
        fs = [torch.as_tensor(I.sources(dtype=np.complex64, nrhs=nrhs), device=dev).to(dtype) for I in insts]
        us = [torch.empty((nrhs, I.x.shape[0]), dtype=dtype, device=dev) for I in insts]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(max(warmup, 1)):
                batch.forward(fs, us, stream=side)
            evs = []
            for _ in range(steps):
                flush_l2(flush)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(side)
                batch.forward(fs, us, stream=side)
                b.record(side)
                evs.append((a, b))
        side.synchronize()
        out[prec] = {"ms": float(np.mean([a.elapsed_time(b) for a, b in evs])),
                     "us": [u.to(torch.complex128) for u in us], "status": batch.device_status(),
                     "flops": sum(p.info()["flops_fwd"] for p in plans) * nrhs,
                     "alg_flops": sum(p.info()["jobs_fwd"] for p in plans) * 2 * insts[0].p ** 3 * 8.0 * nrhs,
                     "smem_kb": plans[0].info()["smem_kb"], "steps": steps,
                     "stages_per_launch": plans[0].info()["stages_per_launch"]}
        del batch, plans, fs, us
    u64 = out["fp64"]["us"]
    res = {"fp64_batch_ms": out["fp64"]["ms"], "fp64_status": out["fp64"]["status"]}
    for prec in precisions:
        o = out[prec]
        num = sum(torch.linalg.norm(a - b).item() ** 2 for a, b in zip(o["us"], u64))
        den = sum(torch.linalg.norm(b).item() ** 2 for b in u64)
        worst = max((torch.linalg.norm(a[r] - b[r]) / torch.linalg.norm(b[r])).item()
                    for a, b in zip(o["us"], u64) for r in range(a.shape[0]))
        ms = o["ms"]
        res[prec] = {"ms": ms, "speedup_vs_fp64": out["fp64"]["ms"] / ms,
                     "rel_l2_vs_fp64": (num / den) ** 0.5, "worst_instance_rhs_rel_l2": worst,
                     "gate_1e-6_met": (num / den) ** 0.5 <= 1e-6,
                     "recursive_executed_tflops": o["flops"] / (ms * 1e-3) / 1e12,
                     "recursive_alg_tflops": o["alg_flops"] / (ms * 1e-3) / 1e12,
                     "status": o["status"], "smem_kb": o["smem_kb"], "steps": o["steps"],
                     "stages_per_launch": o["stages_per_launch"]}
    return res


def batch_summary(args, dev, flush):
    """The batched workload as part of the default run: 64 star-curve instances
    (N log-uniform in [512, 16384], as drawn), p = 7, 16 complex64 right-hand sides each."""
    from paper_0801_1524_gb300 import workloads as w
    insts = w.star_batch(nrhs=16)
    r = run_batch(insts, 16, steps32=10, steps64=2, warmup=2, dev=dev, flush=flush,
                  precisions=("fp32", "fp32g", "tc"))
    r["workload"] = ("star_batch: 64 instances, N log-uniform in 512..16384 (sum N = %.0f), p=7, "
                     "16 complex64 RHS each, graph replay; FP32 (paired FP32 multiply-adds), FP32G (the same with "
                     "right-hand sides in groups of eight) and TC (tensor cores, TF32 x 4) batches against the "
                     "FP64 batch" % sum(I.N for I in insts))
    for prec in ("fp32", "fp32g", "tc"):
        r[prec]["instance_rhs_per_s"] = len(insts) * 16 * 1e3 / r[prec]["ms"]
    return r


def p9_rows(dev):
    """p = 9 companion rows, where the paper's error (Tables 1, 3: about 5e-8 in 2D, 3e-7 in
    3D) is below 1e-6, so that the path can be compared with the direct sum itself:
    curve8192 at p = 9 (FP32 and FP64) and sphere128 at p = 9 (FP32; 3D p = 9 has no FP64
    kernel), each against the FP64 GPU direct sum over all targets."""
    import torch
    from paper_0801_1524_gb300 import workloads as w
    from paper_0801_1524_gb300.plan import Plan
    rows = {}
    for inst, precs in ((w.curve8192(p=9), ("fp32", "fp64")), (w.sphere128(p=9), ("fp32",))):
        f = torch.as_tensor(inst.sources()[0], device=dev)
        # the FP64 direct sum does not depend on p: in 3D it comes from a p = 5 FP64 plan of
        # the same points (3D p = 9 has no FP64 kernel)
        ref_plan = Plan(inst.x, inst.k, inst.N, inst.p if "fp64" in precs else 5, precision="fp64")
        exact = ref_plan.direct(f)
        torch.cuda.synchronize()
        row = {"N": int(inst.N), "p": 9, "dim": inst.dim, "nx": int(inst.x.shape[0]), "nk": int(inst.k.shape[0])}
        for prec in precs:
            plan = ref_plan if prec == "fp64" else Plan(inst.x, inst.k, inst.N, inst.p, precision=prec)
            fin = f if prec == "fp64" else f.to(torch.complex64)
            for _ in range(3):
                u = plan.forward(fin)
            evs = []
            for _ in range(10):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                u = plan.forward(fin)
                b.record()
                evs.append((a, b))
            torch.cuda.synchronize()
            err = (torch.linalg.norm(u.to(torch.complex128) - exact) / torch.linalg.norm(exact)).item()
            row[prec] = {"ms": float(np.mean([a.elapsed_time(b) for a, b in evs])),
                         "rel_l2_vs_direct_fp64": err, "le_1e-6": err <= 1e-6}
        rows[inst.name] = row
        del ref_plan
    return rows


def main_batch(args):
    """64 star-curve instances (N log-uniform in [512, 16384], as drawn), p = 7, nrhs
    complex64 right-hand sides each, one graph replay per step."""
    import torch
    from paper_0801_1524_gb300 import workloads as w
    from paper_0801_1524_gb300.plan import Plan
    args.nrhs = args.nrhs or 16
    insts = w.star_batch(nrhs=args.nrhs)
    dev = torch.device("cuda", 0)
    smem_kb, stages, tuned = 0, 0, None
    precs = tuple(args.precision.split(","))
    if args.autotune:  # one configuration for the whole batch, tuned on its largest instance
        big = max(insts, key=lambda I: I.N)
        t0 = time.perf_counter()
        info = Plan(big.x, big.k, big.N, big.p, max_nrhs=args.nrhs, autotune=True).info()
        names = {0: "fp64", 1: "fp32", 2: "tc"}
        prec = "fp32g" if info["rhs_groups"] else names[info["prec"]]
        smem_kb, stages, precs = info["smem_kb"], info["stages_per_launch"], (prec,)
        tuned = {"smem_kb": smem_kb, "stages_per_launch": stages, "precision": precs[0],
                 "tuned_on": f"largest instance (N = {big.N:.0f})", "tuning_s": time.perf_counter() - t0}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    r = run_batch(insts, args.nrhs, args.steps, max(3, min(args.steps, 10)), args.warmup, dev, flush,
                  smem_kb=smem_kb, precisions=precs, stages=stages)
    ms = r[precs[0]]["ms"]
    pairs = sum(I.x.shape[0] * I.k.shape[0] for I in insts) * args.nrhs
    line = {"metric": METRIC + " (batched)", "value": len(insts) * args.nrhs * 1e3 / ms,
            "unit": "instance-RHS transforms/s", "ms_per_step": ms, "steps": args.steps,
            "warmup": args.warmup, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"star_batch: 64 instances, N log-uniform in 512..16384, p=7, "
                                   f"{args.nrhs} complex64 RHS, graph replay",
                       "sum_N": float(sum(I.N for I in insts)),
                       "l2": "flushed between steps (256 MB written, then read back)",
                       "points": int(sum(I.x.shape[0] + I.k.shape[0] for I in insts))},
            "effective_IJ_per_s": pairs * 1e3 / ms, "autotuned": tuned}
    line.update(r)
    return line


def main():
    args = parse()
    if args.workload == "star_batch":
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps(main_batch(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "bfly":
        import __graft_entry__
        __graft_entry__.build()
    if world > 1 and args.impl == "bfly":
        import torch
        import torch.distributed as tdist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group(backend)
        dist = tdist
    if args.impl == "reference":
        line = main_reference(args, rank)
    else:
        line = main_bfly(args, rank, world, dist)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
