#!/usr/bin/env python
"""Benchmark of the GB300 MCM / S-DP solvers.

Headline (one step = one solve of the whole MCM hot path): the 4096-matrix
chain with dims uniform in [1, 32] (seed 1), int32 costs, int16 split table,
one mcm_solve call per step with inputs resident in device memory; the metric
is split evaluations per second, (n^3 - n) / 6 of them per solve.  L2 is
flushed (a 256 MiB write) between timed steps, outside the timed events.

Also printed in the same JSON line:
  e2e          the same solve through mcm_solve_host (host buffers; the copy
               of p in and of m and s out are inside the timed region);
  roofline     the MCM kernel's INT32 issue rate against the ALU peak
               measured in the same run (SM count x INT32 lanes/clk/SM from
               the library's throughput probe x max SM clock; 3 integer ops
               per split evaluation), from CUDA events around each launch;
  cpu_baseline the CPU oracle (single thread) on a bounded sample;
  sdp          the 2^26-cell S-DP table, 32 offsets in [1024, 8192] (seed 2),
               both operators: cells/s and HBM GB/s;
  batched      10,000 chains, n log-uniform in [8, 512], dims U[1, 1000], int64
               (seed 3): one graph-captured persistent launch vs a plain loop
               of one mcm_solve per chain;
  serve        a Poisson request trace (80 % MCM n in [16, 2048] int64, 20 %
               S-DP n in [2^16, 2^24], 16 offsets in [64, 4096], min) through
               the continuous-batching server: p50 / p99 latency and
               throughput vs a plain sequential solve loop.

--impl reference times the CPU oracle (the only reference this project has)
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_MCM = 4096
EVALS_4096 = (N_MCM ** 3 - N_MCM) // 6
METRIC = "MCM split-evals/s (n=4096, batched) vs plain; S-DP cells/s; served p99 latency"
INT_OPS_PER_EVAL = 3          # weight multiply-add, second add, min


def _rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# ---------------------------------------------------------------------------
# clock sampling (nvidia-smi during the timed region)
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        return time.time()

    def stop(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, samples = [], [], set(), 0
        for ts, line in self.lines:
            if not (t0 - 0.15 <= ts <= t1 + 0.15):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            samples += 1
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                pass
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                 parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": samples}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def measure_int32_peak(lib, native, stream):
    """The INT32 roofline's denominator, measured on this GPU by the
    library's throughput probe (dp_measure_int32_rates): SM count from the
    device, lanes per clock per SM from dependency chains of one instruction
    kind counted in SM cycles.  The peak is the combined rate of both integer
    pipes (two-input adds, which the compiler spreads over the ALU and FMA
    pipes) at the maximum SM clock."""
    out = (ctypes.c_double * 10)()
    native.check(lib.dp_measure_int32_rates(out, 10, ctypes.c_void_p(stream.cuda_stream)))
    rec = {"sms": int(out[6]),
           "lanes_per_clk_sm": {"add3_alu_pipe": round(out[0], 2), "imad_fma_pipe": round(out[1], 2),
                                "min3_alu_pipe": round(out[2], 2), "add2_both_pipes": round(out[3], 2),
                                "add3_imad_interleaved": round(out[4], 2)},
           "bulk_loop_split_evals_per_clk_sm": round(out[5], 3),
           "bulk_loop_i64_split_evals_per_clk_sm": round(out[9], 3),
           "probe_clock_mhz": round(out[7], 1), "max_sm_clock_mhz": out[8]}
    rec["peak_tops"] = rec["sms"] * out[3] * out[8] * 1e6 / 1e12
    rec["bulk_loop_ceiling_tops"] = INT_OPS_PER_EVAL * rec["sms"] * out[5] * out[8] * 1e6 / 1e12
    return rec


def _int32_roofline(kernel_ms, evals, probe, clocks=None, name="mcm_main_kernel<int32>"):
    achieved = INT_OPS_PER_EVAL * evals / (kernel_ms / 1e3) / 1e12
    lanes = probe["lanes_per_clk_sm"]["add2_both_pipes"]
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(probe["peak_tops"], 3),
            "unit": "Tops/s (INT32)", "frac": round(achieved / probe["peak_tops"], 4),
            "kernel": name, "kernel_ms": round(kernel_ms, 4),
            "peak_basis": (f"measured: {probe['sms']} SMs (device) x {lanes:.1f} INT32 lanes/clk/SM "
                           f"(two-input add probe, both integer pipes) x {probe['max_sm_clock_mhz']:.0f} MHz "
                           "(max SM clock)"),
            "frac_of_bulk_loop_ceiling": round(achieved / probe["bulk_loop_ceiling_tops"], 4)}
    if clocks and clocks.get("sm_mhz"):
        roof["frac_at_run_clock"] = round(achieved / (probe["peak_tops"] * clocks["sm_mhz"]
                                                      / probe["max_sm_clock_mhz"]), 4)
    return roof

def _kernel_source_sha():
    h = hashlib.sha256()
    for f in ["mcm.cu", "mcm_kernels.cuh", "dp_common.cuh"]:
        h.update(open(os.path.join(ROOT, "paper_2008_01938_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _profile_traffic():
    """DRAM bytes per launch of the MCM kernel from the machine-readable record
    of the last ncu capture, valid only if it was taken on the current kernel
    source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_records.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get("mcm_main_kernel<int32, unweighted>, n = 4096")
    if not rec or rec.get("kernel_source_sha") != _kernel_source_sha():
        return None
    return float(rec["dram_bytes_per_launch"])


def max_over_ranks(ms, device=None):
    """The largest per-rank step time (ms) over the process group; the local
    value when no group is initialised.  Replicas of the solve run one per
    rank with no exchange, so this is the only collective of the benchmark."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, ms, evals=EVALS_4096):
    """Whole-job split-evals/s of `world` replicas that each solved one chain
    in at most `ms` milliseconds."""
    return world * evals / (ms / 1e3)


def _cpu_baseline(n_sample=2048):
    import oracle
    from paper_2008_01938_gb300 import inputs
    p = inputs.mcm_big()[: n_sample + 1]
    oracle.build()
    t0 = time.perf_counter()
    oracle.mcm(p)
    dt = time.perf_counter() - t0
    ev = (n_sample ** 3 - n_sample) // 6
    return {"value": ev / dt, "unit": "split-evals/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n_sample} matrices of the 4096-matrix chain ({ev} split-evals), "
                      f"single-threaded C oracle, {dt:.2f} s"}


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------
def run_gb300(args):
    import numpy as np
    import torch

    rank, world, local = _rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    import paper_2008_01938_gb300 as dp
    from paper_2008_01938_gb300 import inputs, native
    lib = native.load()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    p_h = inputs.mcm_big()
    p = torch.from_numpy(p_h).to(dev)
    m = torch.empty((N_MCM, N_MCM), dtype=torch.int32, device=dev)
    s = torch.empty((N_MCM, N_MCM), dtype=torch.int16, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        dp.mcm_solve(p, "i32", m, s)
    dp.sync_status()
    probe = measure_int32_peak(lib, native, stream)
    args.probe = probe

    sampler = ClockSampler(local)
    barrier()
    t_wall0 = time.time()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    lib.dp_profile_begin()
    for i in range(args.steps):
        flush.fill_(i)
        starts[i].record(stream)
        dp.mcm_solve(p, "i32", m, s)
        ends[i].record(stream)
    barrier()
    kms, kn, sms_, sn = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    native.check(lib.dp_profile_end(ctypes.byref(kms), ctypes.byref(kn), ctypes.byref(sms_), ctypes.byref(sn)))
    t_wall1 = time.time()
    dp.sync_status()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = max_over_ranks(statistics.mean(step_ms), device=dev)
    clocks = sampler.stop(t_wall0, t_wall1)
    value = replica_throughput(world, ms)
    kernel_ms = kms.value / max(kn.value, 1)

    # correctness spot check of the timed output (cheap: final cell + digest)
    gold = os.path.join(ROOT, "tests", "golden", "fullsize.json")
    parity = None
    if os.path.exists(gold):
        g = json.load(open(gold))["mcm_n4096_seed1"]
        mh = m.cpu().numpy()
        parity = hashlib.sha256(mh.astype("<i4").tobytes()).hexdigest() == g["m_sha256"]

    # e2e through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        ph = torch.from_numpy(p_h).pin_memory()
        mh_t = torch.empty((N_MCM, N_MCM), dtype=torch.int32).pin_memory()
        sh_t = torch.empty((N_MCM, N_MCM), dtype=torch.int16).pin_memory()
        sp = ctypes.c_void_p(stream.cuda_stream)
        native.check(lib.mcm_solve_host(ctypes.c_void_p(ph.data_ptr()), N_MCM, native.DP_COST_I32,
                                        ctypes.c_void_p(mh_t.data_ptr()), ctypes.c_void_p(sh_t.data_ptr()), sp))
        e2e_steps = max(3, min(args.steps, 20))
        barrier()
        e2e_s = 0.0
        for _ in range(e2e_steps):
            flush.fill_(1)           # L2 flush, finished before the timed call starts
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            native.check(lib.mcm_solve_host(ctypes.c_void_p(ph.data_ptr()), N_MCM, native.DP_COST_I32,
                                            ctypes.c_void_p(mh_t.data_ptr()), ctypes.c_void_p(sh_t.data_ptr()), sp))
            e2e_s += time.perf_counter() - t0
        barrier()
        e2e_s /= e2e_steps
        direct = bool(lib.dp_test_host_range_device_address(ctypes.c_void_p(mh_t.data_ptr()),
                                                           mh_t.numel() * 4, 1))
        e2e_parity = (None if parity is None else
                      hashlib.sha256(mh_t.numpy().astype("<i4").tobytes()).hexdigest() == g["m_sha256"])
        e2e = {"value": world * EVALS_4096 / e2e_s, "unit": "split-evals/s",
               "h2d_bytes_per_step": (N_MCM + 1) * 4, "d2h_bytes_per_step": N_MCM * N_MCM * (4 + 2),
               "ms_per_step": e2e_s * 1e3, "parity_sha256_ok": e2e_parity,
               "d2h": ("kernel stores into the pinned host tables" if direct
                       else "copy after the solve"),
               "note": "wall clock of the mcm_solve_host call alone (it returns after the tables are in host "
                       "memory); the L2 flush before each call is outside the timed region"}

    roof = _int32_roofline(kernel_ms, EVALS_4096, probe, clocks)
    roof["traffic"] = _profile_traffic()
    roof["probe"] = probe

    out = {
        "metric": METRIC, "value": value, "unit": "split-evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "MCM n=4096 chain, dims U[1,32] seed 1, int32 m + int16 s, one mcm_solve per step",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks, "e2e": e2e, "roofline": roof, "parity_sha256_ok": parity,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = _cpu_baseline()
    if world == 1 and not args.no_extras:
        extras = set(args.extras.split(","))
        if "sdp" in extras:
            out["sdp"] = bench_sdp(dp, native, lib, dev, args)
        if "small" in extras:
            out["small"] = bench_small(dp, native, lib, dev, args)
        if "interval" in extras:
            out["interval"] = bench_interval(dp, native, lib, dev, args)
        if "batched" in extras:
            out["batched"] = bench_batched(dp, native, lib, dev, args)
        if "serve" in extras:
            out["serve"] = bench_serve(dp, native, dev, args)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def bench_sdp(dp, native, lib, dev, args):
    import numpy as np
    import torch
    from paper_2008_01938_gb300 import inputs
    big = inputs.sdp_instance_big()
    a1 = int(big.offsets[0])
    res = {"workload": "S-DP n=2^26 uint32, k=32 offsets in [1024,8192] (a_1=8192, a_k=1024), preset seed 2"}
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6683.8) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6683.8
    st0 = np.zeros(big.n, dtype=np.uint32)
    st0[:a1] = big.preset
    t = torch.from_numpy(st0.view(np.int32)).to(dev)
    for op in ("min", "add"):
        dp.sdp_solve(t, big.offsets, op=op)
        dp.sync_status()
        reps = 3
        lib.dp_profile_begin()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            dp.sdp_solve(t, big.offsets, op=op)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / reps
        a, b, c, d = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
        native.check(lib.dp_profile_end(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
        kms = c.value / max(d.value, 1)
        cells = big.n - a1
        bytes_ = 4 * cells + 4 * a1
        k = int(big.offsets.size)
        # one SM: 32 shared-memory words per clock at the max SM clock, G words/s
        smem_peak = 32 * args.probe["max_sm_clock_mhz"] * 1e6 / 1e9
        res[op] = {"cells_per_s": cells / (kms / 1e3), "kernel_ms": kms, "wall_ms": wall * 1e3,
                   "roofline": {"bound": "hbm", "achieved": bytes_ / (kms / 1e3) / 1e9, "peak": hbm,
                                "unit": "GB/s", "frac": bytes_ / (kms / 1e3) / 1e9 / hbm,
                                "note": "the shared-memory reads of the recurrence steps bound it, not HBM "
                                        "(smem_roofline)"}}
        av = np.ascontiguousarray(big.offsets.astype(np.int32))
        hook = lib.dp_test_sdp_jump_chunks if op == "add" else lib.dp_test_sdp_min_jump_chunks
        chunks = hook(big.n, ctypes.c_void_p(av.ctypes.data), int(av.size))
        if chunks >= 2:
            algebra = ("products modulo the characteristic polynomial over Z/2^32" if op == "add" else
                       "Boolean products modulo the characteristic polynomial (bitsets) and range minima")
            res[op]["path"] = (f"chunks from jumped windows: {chunks} chunks side by side, their windows from "
                               f"{algebra} (time covers the whole path)")
            nsm = min(chunks, args.probe["sms"])
            peak_w = nsm * smem_peak
            res[op]["smem_roofline"] = {"bound": f"shared memory of the {nsm} SMs the chunks run on",
                                        "achieved": cells * k / (kms / 1e3) / 1e9, "peak": peak_w,
                                        "unit": "G words/s", "frac": cells * k / (kms / 1e3) / 1e9 / peak_w,
                                        "per_unit": f"{k} window reads per cell; the time also covers the "
                                                    "windows' set-up launches"}
        else:
            res[op]["path"] = "step by step on one SM"
            res[op]["smem_roofline"] = {"bound": "shared memory of the one SM the chain runs on",
                                        "achieved": cells * k / (kms / 1e3) / 1e9, "peak": smem_peak,
                                        "unit": "G words/s", "frac": cells * k / (kms / 1e3) / 1e9 / smem_peak,
                                        "per_unit": f"{k} window reads per cell"}
    # the paper's worst case for its pipeline (Section III-A): 32 consecutive
    # offsets, here 1055 .. 1024 (same W = 1024 cells per step, same k)
    cons = np.arange(1055, 1023, -1, dtype=np.int32)
    st1 = np.zeros(big.n, dtype=np.uint32)
    st1[:1055] = inputs.SplitMix64(6).u32(1055)
    t1 = torch.from_numpy(st1.view(np.int32)).to(dev)
    dp.sdp_solve(t1, cons, op="min")
    dp.sync_status()
    lib.dp_profile_begin()
    torch.cuda.synchronize()
    for _ in range(3):
        dp.sdp_solve(t1, cons, op="min")
    torch.cuda.synchronize()
    a, b, c, d = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    native.check(lib.dp_profile_end(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    kms = c.value / max(d.value, 1)
    res["consecutive_min"] = {"workload": "same n, k=32 consecutive offsets 1055..1024 (the paper's conflict worst "
                                          "case), preset seed 6", "cells_per_s": (big.n - 1055) / (kms / 1e3),
                              "kernel_ms": kms,
                              "path": ("chunks from jumped windows" if lib.dp_test_sdp_min_jump_chunks(
                                  big.n, ctypes.c_void_p(cons.ctypes.data), int(cons.size)) >= 2
                                  else "step by step on one SM")}
    return res


def bench_interval(dp, native, lib, dev, args):
    """Interval DP with a per-cell weight on the 4096-cell optimal-BST
    instance: same table size and split count as the MCM headline, with the
    weight table read from HBM and no rank-1 term."""
    import numpy as np
    import torch
    from paper_2008_01938_gb300 import inputs
    inst = inputs.interval_obst(N_MCM, 4, seed=5)
    p = torch.from_numpy(inst.p).to(dev)
    w = torch.from_numpy(inst.w.astype(np.int32)).to(dev)
    m = torch.empty((N_MCM, N_MCM), dtype=torch.int32, device=dev)
    s = torch.empty((N_MCM, N_MCM), dtype=torch.int16, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        dp.interval_dp_solve(p, w, "i32", m, s)
    dp.sync_status()
    reps = 20
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    torch.cuda.synchronize()
    lib.dp_profile_begin()
    for i in range(reps):
        flush.fill_(i)
        starts[i].record(stream)
        dp.interval_dp_solve(p, w, "i32", m, s)
        ends[i].record(stream)
    torch.cuda.synchronize()
    kms, kn, a, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    native.check(lib.dp_profile_end(ctypes.byref(kms), ctypes.byref(kn), ctypes.byref(a), ctypes.byref(b)))
    dp.sync_status()
    ms = statistics.mean(x.elapsed_time(y) for x, y in zip(starts, ends))
    kernel_ms = kms.value / max(kn.value, 1)
    gold = os.path.join(ROOT, "tests", "golden", "fullsize.json")
    parity = None
    if os.path.exists(gold):
        g = json.load(open(gold)).get("interval_obst_n4096_seed5")
        if g:
            parity = hashlib.sha256(m.cpu().numpy().astype("<i4").tobytes()).hexdigest() == g["m_sha256"]
    return {"workload": "interval DP, optimal-BST shape, 4096 cells (4095 keys), key / gap frequencies "
                        "U[1,4] / U[0,4] seed 5, int32 weights, m and s",
            "split_evals_per_s": EVALS_4096 / (ms / 1e3), "ms_per_solve": ms, "main_kernel_ms": kernel_ms,
            "launches_per_solve": 3,
            "roofline": _int32_roofline(kernel_ms, EVALS_4096, args.probe, name="mcm_main_kernel<int32, weighted>"),
            "parity_sha256_ok": parity, "l2": "flushed between solves (outside the timed events)"}


def bench_small(dp, native, lib, dev, args):
    """Latency of the 128-matrix chain (dims U[1,32], seed 0): 127
    tile-diagonal cells in 4 tile-diagonals, far from any throughput bound."""
    import torch
    from paper_2008_01938_gb300 import inputs
    p = torch.from_numpy(inputs.mcm_small()).to(dev)
    m = torch.empty((128, 128), dtype=torch.int32, device=dev)
    s = torch.empty((128, 128), dtype=torch.int16, device=dev)
    for _ in range(10):
        dp.mcm_solve(p, "i32", m, s)
    dp.sync_status()
    reps = 200
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a_, b_ in ev:
        a_.record(stream)
        dp.mcm_solve(p, "i32", m, s)
        b_.record(stream)
    torch.cuda.synchronize()
    dp.sync_status()
    t = sorted(a_.elapsed_time(b_) for a_, b_ in ev)
    evals = (128 ** 3 - 128) // 6
    return {"workload": "MCM n=128 chain, dims U[1,32] seed 0, int32, one mcm_solve (prologue + main kernel)",
            "median_us": t[reps // 2] * 1e3, "p90_us": t[(9 * reps) // 10] * 1e3,
            "split_evals_per_s": evals / (t[reps // 2] / 1e3)}


def bench_batched(dp, native, lib, dev, args):
    import numpy as np
    import torch
    from paper_2008_01938_gb300 import inputs
    b = inputs.mcm_batch()
    total = int(sum((int(n) ** 3 - int(n)) // 6 for n in b.ns))
    plan = dp.McmPlan(b.ns, cost="i64")
    p_all = torch.from_numpy(b.p_all).to(dev)
    p_off = torch.from_numpy(b.p_off[:-1].copy()).to(dev)
    tab_off = torch.from_numpy(b.tab_off[:-1].copy()).to(dev)
    m_all = torch.empty(int(b.tab_off[-1]), dtype=torch.int64, device=dev)
    s_all = torch.empty(int(b.tab_off[-1]), dtype=torch.int16, device=dev)
    st = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(st):
        tuned = plan.autotune(p_all, p_off, tab_off, m_all, s_all, stream=st)
    st.synchronize()
    dp.sync_status()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        plan.solve(p_all, p_off, tab_off, m_all, s_all, stream=st)
    reps = 10
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    dp.sync_status()
    t_graph = e0.elapsed_time(e1) / reps / 1e3
    # the same plan launched directly on the stream (no graph)
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        e0.record(st)
        for _ in range(reps):
            plan.solve(p_all, p_off, tab_off, m_all, s_all, stream=st)
        e1.record(st)
    torch.cuda.synchronize()
    dp.sync_status()
    t_nograph = e0.elapsed_time(e1) / reps / 1e3
    gold = os.path.join(ROOT, "tests", "golden", "fullsize.json")
    parity = None
    if os.path.exists(gold):
        gg = json.load(open(gold)).get("mcm_batch10000_seed3")
        if gg:
            parity = hashlib.sha256(m_all.cpu().numpy().astype("<i8").tobytes()).hexdigest() == gg["m_sha256_concat"]
    # plain loop: one mcm_solve per chain, same device buffers
    views = [(p_all[int(b.p_off[i]):int(b.p_off[i + 1])], m_all[int(b.tab_off[i]):int(b.tab_off[i + 1])].view(
        int(b.ns[i]), int(b.ns[i])), s_all[int(b.tab_off[i]):int(b.tab_off[i + 1])].view(int(b.ns[i]), int(b.ns[i])))
        for i in range(b.ns.size)]
    for v in views[:50]:
        dp.mcm_solve(v[0], "i64", v[1], v[2])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record()
    for v in views:
        dp.mcm_solve(v[0], "i64", v[1], v[2])
    e1.record()
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    dp.sync_status()
    plan.destroy()
    # roofline: the int64 solver's own bulk loop, measured by the probe (split
    # evaluations per clock per SM at two resident blocks) on every SM at the
    # maximum clock; an int64 split evaluation is several INT32 instructions
    roof = None
    probe = getattr(args, "probe", None)
    if probe and probe.get("bulk_loop_i64_split_evals_per_clk_sm"):
        rate = probe["bulk_loop_i64_split_evals_per_clk_sm"]
        peak = probe["sms"] * rate * probe["max_sm_clock_mhz"] * 1e6
        roof = {"bound": "alu", "achieved": total / t_graph, "peak": peak, "unit": "split-evals/s (int64)",
                "frac": round(total / t_graph / peak, 4), "kernel": "mcm_main_kernel<int64> (graph replay)",
                "peak_basis": (f"measured: {probe['sms']} SMs x {rate:.2f} int64 split evaluations/clk/SM "
                               f"(the int64 solver's bulk loop on a staged panel, 2 blocks/SM) x "
                               f"{probe['max_sm_clock_mhz']:.0f} MHz")}
    return {"workload": "10,000 chains, n log-uniform [8,512], dims U[1,1000] seed 3, int64 costs",
            "roofline": roof,
            "split_evals": total, "graph_evals_per_s": total / t_graph, "graph_ms": t_graph * 1e3,
            "no_graph_ms": t_nograph * 1e3,
            "plain_loop_evals_per_s": total / t_plain, "plain_loop_ms": t_plain * 1e3,
            "speedup_vs_plain": t_plain / t_graph, "parity_sha256_ok": parity,
            "autotuned": {"levels_per_bulk_task": tuned[0], "blocks_per_sm": tuned[1]}}


SERVE_CLASSES = [("mcm", 16, 64), ("mcm", 64, 256), ("mcm", 256, 1024), ("mcm", 1024, 2049),
                 ("sdp", 1 << 16, 1 << 20), ("sdp", 1 << 20, (1 << 24) + 1)]


def _serve_class(r):
    for i, (kind, lo, hi) in enumerate(SERVE_CLASSES):
        if r.kind == kind and lo <= r.n < hi:
            return i
    return -1


def _class_stats(trace, lat_ms):
    """p50 / p99 / max latency (ms) per request class: MCM by n, S-DP by n."""
    import numpy as np
    out = {}
    for i, (kind, lo, hi) in enumerate(SERVE_CLASSES):
        v = np.array([l for r, l in zip(trace, lat_ms) if l is not None and _serve_class(r) == i])
        if v.size:
            out[f"{kind} n in [{lo}, {hi - 1}]"] = {"requests": int(v.size), "p50_ms": float(np.percentile(v, 50)),
                                                     "p99_ms": float(np.percentile(v, 99)), "max_ms": float(v.max())}
    return out


def bench_serve(dp, native, dev, args):
    """The served Poisson trace through the continuous-batching server, and a
    plain sequential loop (one solve at a time, in arrival order) over the
    same trace.  The plain loop's service times are measured on a stratified
    sample (every `serve_sample`-th request) and the loop is simulated over
    the whole trace with, for each other request, the measured time of the
    sampled request of the same kind nearest in log n; its latencies include
    the queueing that an arrival rate above its throughput causes."""
    import bisect
    import numpy as np
    import torch
    from paper_2008_01938_gb300 import inputs
    t_gen = time.perf_counter()
    trace = inputs.serve_trace(rate=args.serve_rate, duration=args.serve_seconds, seed=4)
    t_gen = time.perf_counter() - t_gen
    if not trace:
        return None
    srv = dp.Server(hbm_cap_bytes=150 << 30, max_inflight=100000, num_streams=4, max_batch=64, device=dev.index)
    # warm the kernels
    for r in trace[:8]:
        tk = srv.submit_mcm(r.dims) if r.kind == "mcm" else srv.submit_sdp(r.n, r.offsets, r.preset)
        while srv.poll(tk) is None:
            time.sleep(1e-4)
        srv.release(tk)
    t_base = srv.now() + 0.01
    outstanding = {}
    lat = [None] * len(trace)
    busy = 0
    i = 0
    while i < len(trace) or outstanding:
        now = srv.now()
        while i < len(trace) and t_base + trace[i].t_arrival <= now:
            r = trace[i]
            tk = srv.submit_mcm(r.dims) if r.kind == "mcm" else srv.submit_sdp(r.n, r.offsets, r.preset)
            if tk is None:
                busy += 1
                break
            outstanding[tk] = i
            i += 1
        for tk in list(outstanding):
            res = srv.poll(tk)
            if res is not None:
                if res.status != 0:
                    raise RuntimeError(f"request failed with status {res.status}")
                j = outstanding.pop(tk)
                lat[j] = (res.t_done - (t_base + trace[j].t_arrival)) * 1e3
                srv.release(tk)
        time.sleep(2e-5)
    t_end = srv.now()
    srv.close()
    lat_ms = np.array([x for x in lat if x is not None])
    served = {"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
              "max_ms": float(lat_ms.max()), "requests": len(lat_ms),
              "throughput_req_s": len(lat_ms) / (t_end - t_base), "busy_retries": busy,
              "by_class": _class_stats(trace, lat)}
    # plain sequential loop: measured service times on a stratified sample
    step = max(1, args.serve_sample)
    sample = list(range(0, len(trace), step))
    svc = {}
    for j in sample:
        r = trace[j]
        t0 = time.perf_counter()
        if r.kind == "mcm":
            pt = torch.from_numpy(r.dims).to(dev)
            dp.mcm_solve(pt, "i64")
        else:
            st = np.zeros(max(r.n, int(r.offsets[0])), dtype=np.uint32)
            st[: r.offsets[0]] = r.preset
            tt = torch.from_numpy(st.view(np.int32)).to(dev)
            dp.sdp_solve(tt, r.offsets, op="min", n=r.n)
        dp.sync_status()
        svc[j] = time.perf_counter() - t0
    by_kind = {}
    for j in sample:
        by_kind.setdefault(trace[j].kind, []).append((math.log(trace[j].n), svc[j]))
    for k in by_kind:
        by_kind[k].sort()
    def service(j):
        if j in svc:
            return svc[j]
        pts = by_kind[trace[j].kind]
        x = math.log(trace[j].n)
        q = bisect.bisect_left(pts, (x, -1.0))
        cand = [pts[c] for c in (q - 1, q) if 0 <= c < len(pts)]
        return min(cand, key=lambda p: abs(p[0] - x))[1]
    fin, lats = 0.0, []
    for j, r in enumerate(trace):
        start = max(r.t_arrival, fin)
        fin = start + service(j)
        lats.append((fin - r.t_arrival) * 1e3)
    lats_a = np.array(lats)
    plain = {"p50_ms": float(np.percentile(lats_a, 50)), "p99_ms": float(np.percentile(lats_a, 99)),
             "requests": len(trace), "throughput_req_s": len(trace) / fin if fin > 0 else None,
             "by_class": _class_stats(trace, lats),
             "method": (f"one solve at a time in arrival order; service times measured on every {step}th request "
                        f"({len(sample)} solves), the others take the time of the sampled request of the same kind "
                        "nearest in log n; queueing simulated over the whole trace")}
    return {"workload": f"Poisson {args.serve_rate:.0f} req/s for {args.serve_seconds:.0f} s (seed 4): 80% MCM "
                        f"n log-U[16,2048] int64, 20% S-DP n log-U[2^16,2^24] k=16 min; cap 150 GB",
            "trace_generation_s": t_gen, "served": served, "plain_sequential_loop": plain}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------
def run_reference(args):
    rank, world, local = _rank()
    if rank != 0:
        return
    import oracle
    from paper_2008_01938_gb300 import inputs
    oracle.build()
    n_s = 384
    p = inputs.mcm_big()[: n_s + 1]
    ev = (n_s ** 3 - n_s) // 6
    for _ in range(args.warmup):
        oracle.mcm(p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.mcm(p)
    dt = (time.perf_counter() - t0) / args.steps
    value = ev / dt
    sample = f"first {n_s} matrices of the 4096-matrix chain ({ev} split-evals) per step, single-threaded C oracle"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "split-evals/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": "MCM n=4096 chain, dims U[1,32] seed 1 (bounded sample per step)"},
           "cpu_baseline": {"value": value, "unit": "split-evals/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "split-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--extras", default="small,sdp,interval,batched,serve",
                    help="comma-separated sections after the headline: small, sdp, interval, batched, serve")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-sample", type=int, default=40,
                    help="the plain loop's service times are measured on every n-th request of the trace")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
