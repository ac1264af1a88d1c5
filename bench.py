#!/usr/bin/env python
"""Benchmark: permuted statistics per second of the efficient permutation test.

A step is one whole permutation test (block build, relabeling draws, contraction,
combination, p-value) on the high-dimensional ED workload: nx = 2000, ny = 3000,
p = 1000, Y mean 0.05 on the first 50 coordinates, B = 10000 permutations.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is permuted statistics per second with the
inputs already in device memory (each step timed with CUDA events; the L2 cache is
flushed between steps by writing a 256 MiB buffer); `e2e` is the same metric through
the C ABI with pinned host buffers, host<->device copies inside the timed region.
With N > 1 (torchrun) every rank runs its own independent test (replicas, weak
scaling); value = all ranks' permuted statistics / the slowest rank's time.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "permuted stats/s & p99 test latency, tuned vs plain FP32 GPU at rel err ≤1e-5"
UNIT = "permuted stats/s"
KERNELS_PER_STEP = 13  # libept kernels launched by one ept_test call (split-BF16 path)
# dram read + write bytes of one k_contract_tc launch on the highdim workload, from the ncu
# capture summarised in profiles/k_contract_tc_highdim_ed.md (None once the kernel changes)
CONTRACT_TRAFFIC = {"highdim": 64.42e6}  # k_contract_tc unchanged since that capture


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="highdim", choices=["highdim", "mmd", "small"])
    ap.add_argument("--plain-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="run only --warmup + 1 tuned steps (a short program to capture under ncu)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _spec(name):
    from paper_2406_06488_gb300 import workloads
    return workloads.NAMED[name]


def _cpu_baseline(spec, X, Y, budget_s=20.0):
    """The FP64 oracle (direct recomputation of each permuted statistic from the
    permuted raw rows, Algorithm 4), timed on a bounded sample of relabelings."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    sel = oracle.perm_select(spec.seed, spec.nx, spec.ny, 1, 64)
    t0 = time.perf_counter()
    done = 0
    vals = []
    while done < 64:
        vals.append(oracle.stat_select(X, Y, sel[done], spec.stat, spec.sigma))
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d relabelings (draws 1..%d) of the %s workload, each statistic recomputed in FP64 from "
                      "the permuted raw rows (Algorithm 4), threads splitting the rows; %.1f s"
                      % (done, done, "ED nx=%d ny=%d p=%d" % (spec.nx, spec.ny, spec.p), dt)}, vals


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2406_06488_gb300 import workloads
    spec = _spec(args.workload)
    X, Y = workloads.gaussian_pair(spec)
    oracle.build()
    cores = oracle.num_threads()
    sel = oracle.perm_select(spec.seed, spec.nx, spec.ny, 1, args.warmup + args.steps)
    for k in range(args.warmup):
        oracle.stat_select(X, Y, sel[k], spec.stat, spec.sigma)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.stat_select(X, Y, sel[args.warmup + k], spec.stat, spec.sigma)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%s: %s nx=%d ny=%d p=%d B=%d" % (args.workload, spec.stat.upper(), spec.nx,
                                                                      spec.ny, spec.p, spec.B),
                       "reference": "FP64 CPU oracle, one permuted statistic per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one relabeling per step (draws %d..%d), direct FP64 recomputation "
                                       "(Algorithm 4)" % (args.warmup + 1, args.warmup + args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept, workloads
    import dataclasses

    spec = _spec(args.workload)
    spec = dataclasses.replace(spec, seed=spec.seed + rank, data_seed=spec.data_seed + rank)
    X, Y = workloads.gaussian_pair(spec)
    ctx = ept.Context(local)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(prec):
        return ctx.test(Xd, Yd, B=spec.B, seed=spec.seed, stat=spec.stat, sigma=spec.sigma, prec=prec)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    if args.profile:
        for _ in range(args.warmup + 1):
            step("split_bf16")
        torch.cuda.synchronize()
        ctx.close()
        return 0

    # ---- tuned path, inputs resident on the device
    for _ in range(args.warmup):
        step("split_bf16")
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    step_ms, contract_ms, masks_ms, build_ms = [], [], [], []
    last = None
    for k in range(args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = step("split_bf16")
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        contract_ms.append(last.ms_contract)
        masks_ms.append(last.ms_masks)
        build_ms.append(last.ms_build)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    tot_ms = sum(step_ms)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([tot_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = spec.B * ws * args.steps / (tot_ms / 1000.0)

    # ---- plain FP32 path (the comparison side of the metric)
    plain_ms = []
    for _ in range(1):
        step("plain_fp32")
    for k in range(args.plain_steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step("plain_fp32")
        e1.record(stream)
        e1.synchronize()
        plain_ms.append(e0.elapsed_time(e1))

    # ---- end to end through the C ABI with pinned host buffers
    Xh = torch.from_numpy(X).pin_memory().numpy()
    Yh = torch.from_numpy(Y).pin_memory().numpy()
    ctx.test(Xh, Yh, B=spec.B, seed=spec.seed, stat=spec.stat, sigma=spec.sigma, prec="split_bf16")
    e2e_s = []
    for k in range(args.e2e_steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.test(Xh, Yh, B=spec.B, seed=spec.seed, stat=spec.stat, sigma=spec.sigma, prec="split_bf16")
        e2e_s.append(time.perf_counter() - t0)
        _ = r.p_value
    e2e_value = spec.B * ws / statistics.mean(e2e_s)

    if rank != 0:
        ctx.close()
        return 0

    peaks, peak_kind = _peaks()
    n = spec.nx + spec.ny
    pairs = n * (n + 1) // 2
    alg_flops = 2.0 * pairs * (spec.B + 1)
    t_contract = statistics.mean(contract_ms) / 1000.0
    achieved_tflops = alg_flops / t_contract / 1e12
    peak = float(peaks.get("bf16_tflops", 1900.0))
    n_pad = (n + 255) // 256 * 256
    npan = n_pad // 256
    stored = sum((n_pad - 256 * I) * 256 for I in range(npan))
    cols = (spec.B + 1 + 255) // 256 * 256
    mma_flops = 2.0 * 2.0 * stored * cols
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu, _ = _cpu_baseline(spec, X, Y)
    sorted_ms = sorted(step_ms)
    p99 = sorted_ms[min(len(sorted_ms) - 1, int(np.ceil(0.99 * len(sorted_ms))) - 1)]
    psorted = sorted(plain_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "highdim ED test: nx=%d ny=%d p=%d B=%d, X~N(0,I), Y~N(mu,I) mu=0.05 on first 50 "
                               "coords" % (spec.nx, spec.ny, spec.p, spec.B) if args.workload == "highdim"
                   else "%s: %s nx=%d ny=%d p=%d B=%d" % (args.workload, spec.stat, spec.nx, spec.ny, spec.p, spec.B),
                   "precision": "blocks FP32, contraction split-BF16 (hi+lo) on tcgen05, FP32 accumulate, FP64 "
                                "combine", "l2": "flushed between steps (256 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "p50_ms": statistics.median(step_ms), "p99_ms": p99,
        "phase_ms": {"build": statistics.mean(build_ms), "masks": statistics.mean(masks_ms),
                     "contract": statistics.mean(contract_ms)},
        "plain_fp32": {"value": spec.B * ws / (statistics.mean(plain_ms) / 1000.0), "unit": UNIT,
                       "ms_per_step": statistics.mean(plain_ms), "p50_ms": statistics.median(plain_ms),
                       "p99_ms": psorted[-1], "steps": args.plain_steps},
        "roofline": {"bound": "tensor", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / peak, "traffic": CONTRACT_TRAFFIC.get(args.workload),
                     "kernel": "k_contract_tc",
                     "peak_kind": "%s bf16 dense burst" % peak_kind,
                     "algorithmic_flops_per_launch": alg_flops,
                     "mma_flops_per_launch": mma_flops,
                     "mma_frac": mma_flops / t_contract / 1e12 / peak},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int((spec.nx + spec.ny) * spec.p * 4),
                "d2h_bytes_per_step": int((spec.B + 1) * 8 + 48), "steps": args.e2e_steps},
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "clocks": clocks,
        "result": {"observed": last.observed, "p_value": last.p_value, "n_near_tie": last.n_near_tie},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
