"""Benchmark of the HSE Fock-like exchange hot path (one JSON line on rank 0).

A step is one hse_fock_apply over the whole workload: every ordered pair (i, k; j, k') of
the 24^3-grid, 8x8x8 Monkhorst-Pack (512 k-points) silicon-like cell with 16 occupied bands
and 32 target bands (the 16 occupied + 16 empty ones) goes through pair density -> 3-D FFT ->
screened kernel -> inverse FFT -> multiply-accumulate (134,217,728 pair convolutions).  This
is the largest single-GPU configuration of the method's workloads.  Inputs are seeded
synthetic orbitals already resident in HBM; they (2.7 GB) are far larger than L2 (129 MB),
so no flush is needed between steps.  The 20^3, 4x4x4 k, 16-band cell (key "c64_20cube") and
the 32-cell uneven batch, batched call against 32 separate calls (key "batched_32_cells"), are
reported beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl cuda|reference]

Under torchrun each rank runs its own replica of the workload (independent problems,
weak scaling, no data-path collective); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HSE V_xψ orbital-pair convolutions/sec and % roofline at stated err vs FP64"
UNIT = "pair-convolutions/s"
WORKLOAD = 2  # the 24^3 grid, 512 k-point, 16 occupied + 32 target band workload
SECOND = 1    # the 20^3 grid, 64 k-point, 16-band workload (an extra key of the line)
FP32_LANES_PER_SM = 128  # FP32 FMA lanes of an SM (4 schedulers x 32)
DEFAULT_SM_MHZ = 2070.0  # maximum SM clock of a GB300, used when no measured figure exists

# DRAM traffic of one launch of the fused 24^3 kernel from an ncu capture of the full
# workload, valid only while the kernel sources hash to the value recorded with it (else
# reported as null).
TRAFFIC = {"sha": "a6f17334f06074fd", "bytes_per_launch": 115.83e9}  # 106.37 GB read + 9.46 GB written


def _code_only(src: str) -> str:
    """The source without comments and blank lines (what the compiler sees of the kernel).
    Sufficient for these files, whose string literals hold no comment markers."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


KERNEL_SOURCES = ("fft_reg.cuh", "pairconv_c64.cuh", "pairconv_tc.cuh", "tc_dft.cuh", "pairconv_tma.cuh", "tma.cuh",
                  "tmem.cuh", "tmem_gen.cuh", "launch.cuh", "pairconv_24.cu")


def kernel_source_sha() -> str:
    """Hash of the code (comments excluded) of the sources the bench kernel is built from."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1507_05156_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def algorithmic_flops_per_pair(N: int) -> float:
    """10 N log2 N (two 3-D FFTs at 5 N log2 N) + 16 N (pair product 6, kernel 2, MAC 8)."""
    return 10.0 * N * np.log2(N) + 16.0 * N


def fp32_peak_tflops(sms: int, sm_mhz: float) -> float:
    """FP32 ALU peak from unit counts and the clock: SMs x 128 FMA lanes x 2 flop x clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def max_sm_mhz(clocks: dict) -> tuple:
    """(maximum SM clock in MHz, where it came from): nvidia-smi's clocks.max.sm sampled during
    the run, else MEASURED_PEAKS.json's sm_max_mhz, else the GB300's 2070 MHz."""
    if clocks and clocks.get("sm_max_mhz"):
        return float(clocks["sm_max_mhz"]), "nvidia-smi clocks.max.sm during the run"
    m = _measured_peak("sm_max_mhz")
    if m:
        return m, "MEASURED_PEAKS.json sm_max_mhz"
    return DEFAULT_SM_MHZ, "GB300 maximum SM clock (no measured figure)"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cores() -> int:
    return int(os.environ.get("HSE_ORACLE_WORKERS", os.cpu_count() or 1))


def oracle_sample(u_occ, occ, u_tgt, cell, targets, kocc=None):
    """Time the FP64 oracle on a list of (k, i) targets (every k' of the mesh, or the k' of
    kocc); u_occ, u_tgt: complex128 arrays of the values the GPU reads.  Returns (values,
    seconds)."""
    import oracle
    t0 = time.perf_counter()
    ref = oracle.fock_apply(u_occ, occ, u_tgt, cell.kpts, cell.lattice, cell.grid, cell.omega, cell.alpha,
                            targets=targets, kocc=kocc)
    return ref, time.perf_counter() - t0


def sample_targets(cell, count, seed=11):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(cell.nk)), int(rng.integers(cell.n_tgt))) for _ in range(count)]


def sample_kocc(cell, count, seed):
    """`count` distinct k' of the mesh (the partner sample of the reference arm's steps)."""
    rng = np.random.default_rng(seed)
    return sorted(int(k) for k in rng.choice(cell.nk, size=min(count, cell.nk), replace=False))


def rounded_c64(a):
    """complex128 copy of the complex64 values the GPU path reads."""
    return a.astype(np.complex64).astype(np.complex128)


# Reference-arm sample per step: one target (k, i) against every occupied band of
# REF_KPRIME sampled k' (1,024 pair convolutions at 16 bands), about half a second of oracle.
REF_KPRIME = 64


def run_reference(args, rank, world):
    """The oracle on the host cores, each step a bounded sample of the same workload: one
    target orbital against all bands of REF_KPRIME k' of the mesh."""
    if rank != 0:
        return
    from paper_1507_05156_gb300 import inputs
    cell = inputs.workload(WORKLOAD)
    u_occ = rounded_c64(cell.u_occ)
    u_tgt = cell.u_tgt.astype(np.complex64)  # rounded to complex128 by the oracle per target
    for w in range(args.warmup):
        oracle_sample(u_occ, cell.occ, u_tgt, cell, sample_targets(cell, 1, seed=100 + w), sample_kocc(cell, REF_KPRIME, 300 + w))
    times = []
    for s in range(args.steps):
        _, dt = oracle_sample(u_occ, cell.occ, u_tgt, cell, sample_targets(cell, 1, seed=200 + s),
                              sample_kocc(cell, REF_KPRIME, 400 + s))
        times.append(dt)
    pairs = 1 * REF_KPRIME * cell.n_occ
    value = pairs * len(times) / sum(times)
    sample = (f"per step 1 target (k,i) x {REF_KPRIME} sampled k' x {cell.n_occ} bands = {pairs} of the "
              f"{cell.pairs} pair convolutions of the workload")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(cell),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(cell, l2=None):
    nbytes = 8 * cell.npts * cell.nk * (cell.n_occ + cell.n_tgt)
    if l2 is None:
        l2 = (f"not flushed: the inputs ({nbytes / 1e9:.2f} GB of complex64 orbitals) are larger than L2 (129 MB)"
              if nbytes > 256e6 else "flushed between timed steps by a 256 MB write")
    return {"workload": cell.name, "grid": list(cell.grid), "nk": cell.nk, "n_occ": cell.n_occ,
            "n_tgt": cell.n_tgt, "omega": cell.omega, "alpha": cell.alpha, "pairs_per_step": cell.pairs, "l2": l2}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's value (the slowest replica's time); x itself on one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of `world` independent replicas (weak scaling): every rank
    processes units_per_rank in the time of the slowest rank."""
    return world * units_per_rank / seconds


def run_second(dev, steps, warmup, sms, sm_mhz):
    """The 20^3, 4x4x4 k, 16-band cell (1,048,576 pair convolutions): the earlier bench workload,
    reported beside the headline.  Inputs (65.5 MB) fit in L2, so a 256 MB write flushes it
    between steps (outside the events)."""
    import torch
    from paper_1507_05156_gb300 import hse, inputs
    cell = inputs.workload(SECOND)
    plan = hse.get_plan(cell.grid, cell.lattice, cell.kpts, cell.n_occ, cell.n_tgt, cell.omega, cell.alpha)
    u = torch.from_numpy(cell.u_occ.astype(np.complex64)).to(dev)
    occ = torch.from_numpy(cell.occ).to(dev)
    out = torch.empty_like(u)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        hse.hse_fock_apply(plan, u, occ, u, out=out)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        for s in range(steps):
            flush.fill_(s & 0xFF)
            ev[s][0].record(stream)
            hse.hse_fock_apply(plan, u, occ, u, out=out)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    hse.hse_status(plan)
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    flops = algorithmic_flops_per_pair(cell.npts) * cell.pairs
    peak = fp32_peak_tflops(sms, sm_mhz)
    return {"workload": cell.name, "value": cell.pairs / ms * 1e3, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "roofline_frac": flops / ms / 1e9 / peak, "l2": config_dict(cell)["l2"], "clocks": clk.summary()}


def run_batched(dev, steps, warmup, sms, sm_mhz):
    """The 32-cell uneven batch (grids from {12, 16, 18, 20, 24}^3, 2^3-4^3 k, 4-16 bands;
    5,094,023 pair convolutions): one hse_fock_apply_batched call per step (autotuned on its first
    call, then one graph replay), and the same cells as 32 separate hse_fock_apply calls."""
    import torch
    from paper_1507_05156_gb300 import hse, inputs
    stream = torch.cuda.current_stream()
    cells = inputs.batched_cells()
    plan = hse.BatchedPlan(cells)
    uo = [torch.from_numpy(c.u_occ.astype(np.complex64)).to(dev) for c in cells]
    oc = [torch.from_numpy(c.occ).to(dev) for c in cells]
    out = [torch.empty_like(u) for u in uo]
    clk_b, clk_s = {}, {}
    ms = _timed(lambda: hse.hse_fock_apply_batched(plan, uo, oc, uo, out=out), steps, warmup, stream, clk_b)
    hse.hse_status(plan)
    plans = [hse.Plan(c.grid, c.lattice, c.kpts, c.n_occ, c.n_tgt, c.omega, c.alpha) for c in cells]

    def separate():
        for pl, u, o, r in zip(plans, uo, oc, out):
            hse.hse_fock_apply(pl, u, o, u, out=r)

    ms_sep = _timed(separate, steps, warmup, stream, clk_s)
    pairs = sum(c.pairs for c in cells)
    flops = sum(algorithmic_flops_per_pair(int(np.prod(c.grid))) * c.pairs for c in cells)
    peak = fp32_peak_tflops(sms, sm_mhz)
    return {"workload": "batched_32_uneven_cells", "cells": len(cells), "pairs_per_step": pairs,
            "value": pairs / ms * 1e3, "unit": UNIT, "ms_per_step": ms, "steps": clk_b.get("timed_calls", steps),
            "roofline_frac": flops / ms / 1e9 / peak,
            "separate_calls": {"ms_per_step": ms_sep, "value": pairs / ms_sep * 1e3, "batched_speedup": ms_sep / ms,
                               "clocks": clk_s},
            "clocks": clk_b, "l2": "not flushed (one graph replay per step, back to back)"}


def run_cuda(args, rank, world, dist):
    import torch
    from paper_1507_05156_gb300 import hse, inputs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cell = inputs.workload(WORKLOAD)
    d = torch.complex64
    plan = hse.get_plan(cell.grid, cell.lattice, cell.kpts, cell.n_occ, cell.n_tgt, cell.omega, cell.alpha,
                        dtype=d)
    uo_np = cell.u_occ.astype(np.complex64)
    ut_np = cell.u_tgt.astype(np.complex64)
    uo_host = torch.from_numpy(uo_np).pin_memory()
    ut_host = torch.from_numpy(ut_np).pin_memory()
    occ_host = torch.from_numpy(cell.occ).pin_memory()
    u_occ = uo_host.to(dev)
    u_tgt = ut_host.to(dev)
    occ = occ_host.to(dev)
    out = torch.empty_like(u_tgt)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        hse.hse_fock_apply(plan, u_occ, occ, u_tgt, out=out)
    hse.hse_status(plan)

    # ---- device-resident timed region (inputs 2.7 GB > L2: no flush) ------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    l0 = hse.kernel_launches()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            ev[s][0].record(stream)
            hse.hse_fock_apply(plan, u_occ, occ, u_tgt, out=out)
            ev[s][1].record(stream)
        barrier()
    launches = hse.kernel_launches() - l0
    hse.hse_status(plan)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    pairs = cell.pairs
    value = replica_throughput(pairs * args.steps, world, total_ms / 1e3)
    got_rows = None
    if rank == 0 and not args.no_cpu_baseline:
        targets = sample_targets(cell, args.cpu_targets)
        got_rows = np.stack([out[k, i].cpu().numpy() for k, i in targets]).astype(np.complex128)

    # ---- end to end through the public API: pinned host in, host out ------------------
    # Every step copies its inputs (u_occ, u_tgt, occ) from pinned host memory and reads its
    # result back.  The copies run on a second stream into double-buffered device tensors, so
    # step s + 1's upload and step s - 1's download overlap step s's apply.
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    nbuf = min(2, e2e_steps)
    out_host = [torch.empty(out.shape, dtype=d).pin_memory() for _ in range(nbuf)]
    uo_dev = [u_occ] + [torch.empty_like(u_occ) for _ in range(nbuf - 1)]
    ut_dev = [u_tgt] + [torch.empty_like(u_tgt) for _ in range(nbuf - 1)]
    o_dev = [occ] + [torch.empty_like(occ) for _ in range(nbuf - 1)]
    r_dev = [out] + [torch.empty_like(out) for _ in range(nbuf - 1)]
    copy = torch.cuda.Stream(device=dev)
    up_done = [torch.cuda.Event() for _ in range(nbuf)]
    apply_done = [torch.cuda.Event() for _ in range(nbuf)]
    down_done = [torch.cuda.Event() for _ in range(nbuf)]
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy.wait_event(e0)

    def upload(s):
        b = s % nbuf
        with torch.cuda.stream(copy):
            if s >= nbuf:
                copy.wait_event(apply_done[b])  # the apply of step s - nbuf has read this buffer
            uo_dev[b].copy_(uo_host, non_blocking=True)
            ut_dev[b].copy_(ut_host, non_blocking=True)
            o_dev[b].copy_(occ_host, non_blocking=True)
            up_done[b].record(copy)

    upload(0)
    for s in range(e2e_steps):
        b = s % nbuf
        if s + 1 < e2e_steps:
            upload(s + 1)
        stream.wait_event(up_done[b])
        if s >= nbuf:
            stream.wait_event(down_done[b])  # step s - nbuf's result has left this buffer
        hse.hse_fock_apply(plan, uo_dev[b], o_dev[b], ut_dev[b], out=r_dev[b], stream=stream)
        apply_done[b].record(stream)
        with torch.cuda.stream(copy):
            copy.wait_event(apply_done[b])
            out_host[b].copy_(r_dev[b], non_blocking=True)
            down_done[b].record(copy)
    for s in range(max(0, e2e_steps - nbuf), e2e_steps):
        stream.wait_event(down_done[s % nbuf])
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, dist, dev)
    e2e_value = replica_throughput(pairs, world, e2e_ms / 1e3)
    h2d = sum(t.numel() * t.element_size() for t in (uo_host, ut_host, occ_host))
    d2h = out_host[0].numel() * out_host[0].element_size()
    del out_host, uo_dev, ut_dev, o_dev, r_dev

    if rank != 0:
        return

    clocks = clk.summary()
    sm_mhz, mhz_source = max_sm_mhz(clocks)
    peak = fp32_peak_tflops(sms, sm_mhz)

    # ---- the 20^3 cell, reported beside the headline ----------------------------------
    second = None
    if not args.no_second:
        second = run_second(dev, min(args.steps, 20), max(3, args.warmup), sms, sm_mhz)
    batched = None
    if not args.no_batched:
        batched = run_batched(dev, min(args.steps, 5), 2, sms, sm_mhz)

    # ---- the plain FP64 GPU form: every target against a sample of k' (extrapolated) ----
    fp64 = None
    if not args.no_fp64:
        kocc = list(range(args.fp64_kprime))
        plan64 = hse.get_plan(cell.grid, cell.lattice, cell.kpts, cell.n_occ, cell.n_tgt, cell.omega, cell.alpha,
                              dtype=torch.complex128, kocc=kocc)
        u64o = torch.from_numpy(cell.u_occ).to(dev)
        u64t = torch.from_numpy(cell.u_tgt).to(dev)
        o64 = torch.empty_like(u64t)
        hse.hse_fock_apply(plan64, u64o, occ, u64t, out=o64)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hse.hse_fock_apply(plan64, u64o, occ, u64t, out=o64)
        b.record(stream)
        torch.cuda.synchronize()
        hse.hse_status(plan64)
        ms64 = a.elapsed_time(b)
        pairs64 = cell.nk * cell.n_tgt * len(kocc) * cell.n_occ
        rate64 = pairs64 / (ms64 / 1e3)
        fp64 = {"value": rate64, "unit": UNIT, "ms_per_sample": ms64,
                "sample": f"all {cell.nk * cell.n_tgt} targets x {len(kocc)} k' x {cell.n_occ} bands = {pairs64} "
                          f"pair convolutions (down-sampled FP64 plan); full apply extrapolated by pair count",
                "ms_per_step_extrapolated": ms64 * pairs / pairs64,
                "speedup_fused_c64_over_fp64_gpu": value / world / rate64}
        del u64o, u64t, o64, plan64

    # ---- accuracy against the FP64 oracle on sampled targets, and the CPU baseline ----
    cpu = None
    err = None
    if got_rows is not None:
        targets = sample_targets(cell, args.cpu_targets)
        ref, dt = oracle_sample(rounded_c64(cell.u_occ), cell.occ, ut_np, cell, targets)
        err = float(np.linalg.norm(got_rows - ref) / np.linalg.norm(ref))
        cpu_pairs = len(targets) * cell.nk * cell.n_occ
        cpu = {"value": cpu_pairs / dt, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": f"{len(targets)} targets (k,i) x all {cell.nk * cell.n_occ} (k',j) partners"}

    flops = algorithmic_flops_per_pair(cell.npts) * pairs
    kernel_s = (total_ms / args.steps) / 1e3
    achieved = flops / kernel_s / 1e12
    traffic = TRAFFIC["bytes_per_launch"] if TRAFFIC["sha"] == kernel_source_sha() else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(cell),
        "err_vs_fp64": err,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"FP32 FMA lanes x max SM clock ({sms} SMs x {FP32_LANES_PER_SM} x 2 x "
                                    f"{sm_mhz:.0f} MHz, {mhz_source})",
                     "flops_per_launch": flops,
                     "timed": "one hse_fock_apply (the fused kernel and the pencil-blocked relayout of its inputs)"},
        "cpu_baseline": cpu,
        "fp64_gpu": fp64,
        "c64_20cube": second,
        "batched_32_cells": batched,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_profile_case(spec: str):
    """Two applies of one seeded cell (grid side n, n_k^3 Monkhorst-Pack k-points, nb bands,
    complex64; a fourth field "tc" selects the tensor-core option; "batched,C" runs the first C
    cells of the uneven batch instead; "workload,W" the full workload W, u_occ and u_tgt as the
    bench reads them): the launch an ncu capture selects with -s 1 -c 1.  Prints no bench line."""
    import torch
    from paper_1507_05156_gb300 import hse, inputs
    fields = spec.split(",")
    if fields[0] == "workload":  # "workload,W": two applies of the whole workload W
        cell = inputs.workload(int(fields[1]))
        plan = hse.Plan(cell.grid, cell.lattice, cell.kpts, cell.n_occ, cell.n_tgt, cell.omega, cell.alpha)
        uo = torch.from_numpy(cell.u_occ.astype(np.complex64)).cuda()
        ut = torch.from_numpy(cell.u_tgt.astype(np.complex64)).cuda()
        occ = torch.from_numpy(cell.occ).cuda()
        out = torch.empty_like(ut)
        for _ in range(2):
            hse.hse_fock_apply(plan, uo, occ, ut, out=out)
        torch.cuda.synchronize()
        hse.hse_status(plan)
        print(f"profile case {cell.name}: {cell.pairs} pair convolutions per apply", flush=True)
        return
    if fields[0] == "batched":  # "batched,C": two calls on the first C cells of the uneven batch
        cells = inputs.batched_cells(int(fields[1]))
        plan = hse.BatchedPlan(cells)
        uo = [torch.from_numpy(c.u_occ.astype(np.complex64)).cuda() for c in cells]
        oc = [torch.from_numpy(c.occ).cuda() for c in cells]
        out = [torch.empty_like(u) for u in uo]
        for _ in range(2):
            hse.hse_fock_apply_batched(plan, uo, oc, uo, out=out)
        torch.cuda.synchronize()
        hse.hse_status(plan)
        print(f"profile case batched_{len(cells)}: {sum(c.pairs for c in cells)} pair convolutions per call",
              flush=True)
        return
    n, km, nb = (int(x) for x in fields[:3])
    tc = len(fields) > 3 and fields[3] == "tc"
    cell = inputs.make_cell(inputs.SEED_BASE + 100 + n, (n, n, n), (km, km, km), nb, name=f"c64_{n}cube_k{km}_b{nb}")
    u = torch.from_numpy(cell.u_occ.astype(np.complex64)).cuda()
    occ = torch.from_numpy(cell.occ).cuda()
    plan = hse.Plan(cell.grid, cell.lattice, cell.kpts, cell.n_occ, cell.n_tgt, cell.omega, cell.alpha,
                    tensor_cores=tc)
    out = torch.empty_like(u)
    for _ in range(2):
        hse.hse_fock_apply(plan, u, occ, u, out=out)
    torch.cuda.synchronize()
    hse.hse_status(plan)
    print(f"profile case {cell.name}: {cell.pairs} pair convolutions per apply", flush=True)


FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (no measured figure exists for it)


def _measured_peak(key: str):
    """A figure of MEASURED_PEAKS.json at the repository root, or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json"), encoding="utf-8") as fh:
            return float(json.load(fh)[key])
    except (OSError, KeyError, ValueError, TypeError):
        return None
CONFIGS = ("fp64_12cube", "c64_24cube", "c64_24cube_tc", "diff_16cube", "batched")


def _timed(fn, steps, warmup, stream, clocks=None, min_seconds=1.0):
    """Mean milliseconds of fn() over the timed calls after `warmup`, CUDA events on `stream`.
    With a dict `clocks`, nvidia-smi samples the timed region and the dict receives their
    summary and the number of timed calls, which is raised above `steps` where needed so that
    the region lasts at least `min_seconds` (the sampler's 50 ms period sees it)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clocks is not None and min_seconds > 0:
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        steps = max(steps, int(np.ceil(min_seconds * 1e3 / max(a.elapsed_time(b), 1e-3))))
    sampler = ClockSampler(torch.cuda.current_device()) if clocks is not None else None
    if sampler:
        sampler.__enter__()
    try:
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        b.synchronize()
    finally:
        if sampler:
            sampler.__exit__(None, None, None)
    if clocks is not None:
        clocks.update(sampler.summary(), timed_calls=steps)
    return a.elapsed_time(b) / steps


def run_config(name: str, args):
    """One JSON line for another workload of the method (not the headline bench): the plain FP64
    form on the 12^3 cell, the 24^3 cell with 8^3 k-points and 16 + 16 bands, the
    differentiation workload (VJP and backprop through 20 Taylor steps, 16^3, 3^3 k, 8 bands) or
    the 32-cell uneven batch; c64_24cube_tc is the 24^3 workload on the tensor-core option.  Inputs stay on the device; no L2 flush (each call reads far more
    than L2 or is timed back to back, as stated in `config`)."""
    import torch
    from paper_1507_05156_gb300 import hse, inputs, tdks
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    steps, warmup = max(1, args.steps), max(1, args.warmup)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    FP32_PEAK_TFLOPS = fp32_peak_tflops(sms, max_sm_mhz(None)[0])
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic"}
    if name == "batched":
        b = run_batched(dev, steps, warmup, sms, max_sm_mhz(None)[0])
        line.update(value=b["value"], ms_per_step=b["ms_per_step"], steps=b["steps"], warmup=warmup, dtype="f32",
                    config={"workload": b["workload"], "cells": b["cells"], "pairs_per_step": b["pairs_per_step"],
                            "l2": b["l2"]},
                    separate_calls=b["separate_calls"], clocks=b["clocks"],
                    roofline={"bound": "alu", "achieved": b["roofline_frac"] * FP32_PEAK_TFLOPS,
                              "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": b["roofline_frac"],
                              "peak_source": "FP32 FMA lanes x max SM clock"})
    elif name in ("fp64_12cube", "c64_24cube", "c64_24cube_tc"):
        w = 0 if name == "fp64_12cube" else 2
        tc = name == "c64_24cube_tc"
        cell = inputs.workload(w)
        d = torch.complex128 if w == 0 else torch.complex64
        if w == 2:
            steps, warmup = min(steps, 2), 1  # about 9 s per apply
        plan = hse.Plan(cell.grid, cell.lattice, cell.kpts, cell.n_occ, cell.n_tgt, cell.omega, cell.alpha, dtype=d,
                        tensor_cores=tc)
        u_occ = torch.from_numpy(cell.u_occ).to(dev, d)
        u_tgt = torch.from_numpy(cell.u_tgt).to(dev, d)
        occ = torch.from_numpy(cell.occ).to(dev)
        out = torch.empty_like(u_tgt)
        clk = {}
        ms = _timed(lambda: hse.hse_fock_apply(plan, u_occ, occ, u_tgt, out=out), steps, warmup, stream, clk)
        hse.hse_status(plan)
        line["clocks"] = clk
        flops = algorithmic_flops_per_pair(int(np.prod(cell.grid))) * cell.pairs
        peak = FP64_NOMINAL_TFLOPS if w == 0 else FP32_PEAK_TFLOPS
        line.update(value=cell.pairs / ms * 1e3, ms_per_step=ms, steps=clk.get("timed_calls", steps), warmup=warmup,
                    dtype="f64" if w == 0 else "f32",
                    config=dict(config_dict(cell), l2="not flushed" + (" (inputs 2.7 GB > L2)" if w == 2 else "")),
                    roofline={"bound": "alu", "achieved": flops / ms / 1e9, "peak": peak, "unit": "TFLOP/s",
                              "frac": flops / ms / 1e9 / peak,
                              "peak_source": "FP64 nominal" if w == 0 else "FP32 FMA lanes x max SM clock"})
        if tc:
            # executed tensor work: four of the six axis transforms (Y and X, both directions)
            # as (2n)-wide real GEMMs, three split products each, per pair
            n = cell.grid[0]
            tflop = 4 * n * n * 3 * (2 * n) ** 2 * 2 * cell.pairs / ms / 1e9
            peak_tc = _measured_peak("bf16_tflops")
            line["config"]["tensor_cores"] = "Y and X transforms as split-FP16 mma.sync GEMMs"
            line["roofline_alu_algorithmic"] = line["roofline"]
            line["roofline"] = {"bound": "tensor", "achieved": tflop, "peak": peak_tc, "unit": "TFLOP/s",
                                "frac": tflop / peak_tc if peak_tc else None,
                                "peak_source": "measured bf16 dense (FP16 same nominal rate)",
                                "note": "executed FP16 tensor flops of the Y/X GEMMs only"}
    elif name == "diff_16cube":
        cell = inputs.workload(4)
        res, clk = {}, {}
        for d, tag in ((torch.complex64, "c64"), (torch.complex128, "c128")):
            plan = hse.Plan(cell.grid, cell.lattice, cell.kpts, cell.n_occ, cell.n_tgt, cell.omega, cell.alpha,
                            dtype=d)
            u = torch.from_numpy(cell.u_occ).to(dev, d)
            occ = torch.from_numpy(cell.occ).to(dev)
            ybar = (0.5 * u).contiguous()
            out = torch.empty_like(u)
            for key, fn in ((f"apply_ms_{tag}", lambda: hse.hse_fock_apply(plan, u, occ, u, out=out)),
                            (f"vjp_ms_{tag}", lambda: hse.hse_fock_apply_vjp(plan, u, occ, u, ybar)),
                            (f"energy_ms_{tag}", lambda: hse.hse_exchange_energy(plan, u, occ))):
                clk[key] = {}
                res[key] = _timed(fn, steps, warmup, stream, clk[key])
            hse.hse_status(plan)
        # backprop through 20 Taylor steps (dt = 0.02, E = 0.005 along x), checkpointed, complex64
        geom = tdks.Geometry(cell.grid, cell.lattice, cell.kpts, alpha=cell.alpha)
        psi0 = torch.from_numpy(cell.u_occ.astype(np.complex64)).to(dev)
        occ = torch.from_numpy(cell.occ).to(dev)

        def backprop():
            psi = psi0.clone().requires_grad_(True)
            om = torch.tensor(cell.omega, dtype=torch.float64, requires_grad=True)
            out = tdks.propagate(psi, occ, om, geom, 0.02, 20, (0.005, 0.0, 0.0))
            loss = (out.conj() * psi0).real.sum()
            loss.backward()

        clk["backprop_20_steps_ms_c64"] = {}
        res["backprop_20_steps_ms_c64"] = _timed(backprop, 1, 1, stream, clk["backprop_20_steps_ms_c64"])
        # the VJP executes three pair convolutions per pair (one for u_tgt, two for u_occ)
        vflops = 3 * algorithmic_flops_per_pair(int(np.prod(cell.grid))) * cell.pairs
        line["roofline"] = {"bound": "alu", "achieved": vflops / res["vjp_ms_c64"] / 1e9, "peak": FP32_PEAK_TFLOPS,
                            "unit": "TFLOP/s", "frac": vflops / res["vjp_ms_c64"] / 1e9 / FP32_PEAK_TFLOPS,
                            "peak_source": "FP32 FMA lanes x max SM clock",
                            "note": "three executed pair convolutions per pair of the forward"}
        line.update(value=cell.pairs / res["vjp_ms_c64"] * 1e3, ms_per_step=res["vjp_ms_c64"],
                    steps=clk["vjp_ms_c64"].get("timed_calls", steps),
                    warmup=warmup, dtype="f32",
                    config=dict(config_dict(cell), timed="hse_fock_apply_vjp (all three gradients), complex64",
                                l2="not flushed (inputs 7 MB, calls back to back)"),
                    clocks=clk["vjp_ms_c64"], clocks_per_measurement=clk,
                    **{k: round(v, 4) for k, v in res.items()})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--cpu-targets", type=int, default=2, help="oracle targets (full partner sums) for err_vs_fp64")
    ap.add_argument("--e2e-steps", type=int, default=2, help="steps of the end-to-end measurement")
    ap.add_argument("--fp64-kprime", type=int, default=2, help="sampled k' of the FP64 GPU form's timing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-second", action="store_true", help="skip the 20^3 cell reported beside the headline")
    ap.add_argument("--no-batched", action="store_true", help="skip the 32-cell batch reported beside the headline")
    ap.add_argument("--profile-case", default=None, metavar="N,KM,NB[,tc] | batched,C | workload,W",
                    help="only run two applies of one cell (for ncu captures of secondary kernels)")
    ap.add_argument("--config", choices=CONFIGS, default=None,
                    help="time another workload of the method (one JSON line) instead of the bench workload")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.config:
        run_config(args.config, args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    try:
        run_cuda(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
