#!/usr/bin/env python
"""Benchmark: DHT-0 coefficients/s at N = 2^20, eps in {1e-15, 1e-8}, FP64, one GB300.

One step = one discrete Hankel transform of order 0 (Section 6, Eq. 25) at eps = 1e-15 plus
one at eps = 1e-8, each over a batch of ``--nrhs`` seeded standard-normal coefficient
vectors (the paper's Gaussian experiments). value = coefficients transformed / device time.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle instead (direct
O(N^2) FP64 summation on this host's cores) on a bounded sample of rows of the same workload.
Under torchrun each rank runs an independent replica (the transform does not shard across
GPUs here), and the slowest rank's time is reported.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from hankel_inputs import coefficients, sample_rows, seed_for  # noqa: E402

FP64_PEAK_GFLOPS = 152 * 4 * 2.07  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz = 1258 GFLOP/s
HBM_FALLBACK_GBS = 6800.0          # used only when MEASURED_PEAKS.json is absent
FP64_MEASURED_GFLOPS = 1004.0      # DFMA microbenchmark on this part (2 x 502 G instructions/s)
# DRAM bytes per algorithmic byte of a k_fft_pass launch, from an ncu capture of one radix-64
# forward pass over 290 columns of 2^17 points (1167.9 MB measured / 1216.3 MB algorithmic).
FFT_TRAFFIC_RATIO = 1167.9 / 1216.3
METRIC = "DHT-0 coeffs/s at N=2^20 (eps=1e-8,1e-15) served vs plain FP64; p50/p99 ms"
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=2 ** 20)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--eps", default="1e-15,1e-8")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--cpu-rows", type=int, default=1024, help="oracle rows per sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "bench_clocks_%d.csv" % index)

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + CLOCK_FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def cpu_baseline(N, rows_count, seed):
    """Oracle (direct FP64 sum, all host cores) on a bounded sample of DHT rows."""
    import oracle

    c = coefficients("normal", N, 1, seed)[0]
    rows = sample_rows(N, rows_count, seed + 1)
    t0 = time.perf_counter()
    oracle.transform("dht", 0, N, c, rows=rows)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    # one output row costs N J-evaluations; a full transform is N rows, so coefficients/s = rows/s
    return {"value": len(rows) / dt, "unit": "coeffs/s", "cores": cores, "kind": "oracle",
            "sample": "%d of %d rows of one DHT-0 at N=%d (direct O(N^2) FP64 Kahan sum; rows/s = "
                      "coefficients/s of a full transform)" % (len(rows), N, N),
            "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    oracle_dir = os.path.join(ROOT, "oracle")
    if not os.path.isdir(oracle_dir):
        print(json.dumps({"impl": "reference", "unavailable": "oracle sources missing"}))
        return
    N = args.N
    eps = [float(e) for e in args.eps.split(",")]
    times = []
    rows_total = 0
    for step in range(args.warmup + args.steps):
        r = cpu_baseline(N, args.cpu_rows, seed_for(4, step))
        if step >= args.warmup:
            times.append(r["seconds"])
            rows_total += args.cpu_rows
    # the oracle's cost does not depend on eps; one step covers both eps values of the workload
    value = rows_total / sum(times)
    ms_per_step = 1000.0 * len(eps) * N / value
    cores = len(os.sched_getaffinity(0))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "coeffs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "dht0_N%d_eps%s" % (N, "+".join(args.eps.split(","))), "N": N, "eps": eps,
                   "nrhs": 1, "sample_rows_per_step": args.cpu_rows},
        "cpu_baseline": {"value": value, "unit": "coeffs/s", "cores": cores, "kind": "oracle",
                         "sample": "%d seeded rows per step of a DHT-0 at N=%d" % (args.cpu_rows, N)},
        "e2e": {"value": value, "unit": "coeffs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    import paper_1501_01652_gb300 as hk

    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, nrhs = args.N, args.nrhs
    eps_list = [float(e) for e in args.eps.split(",")]
    plans = [hk.Plan("dht", 0, N, e, max_nrhs=nrhs) for e in eps_list]
    c_host = coefficients("normal", N, nrhs, seed_for(4, rank))
    c = torch.from_numpy(c_host).to(dev)
    fs = [torch.empty((nrhs, N), dtype=torch.float64, device=dev) for _ in plans]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    def step():
        for p, f in zip(plans, fs):
            p.exec(c, f, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for p in plans:
        p.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    per_eps_ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in plans] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        wall0 = time.perf_counter()
        for s in range(args.steps):
            flush.zero_()  # evict L2 between timed steps (outside the step events)
            ev[s][0].record(stream)
            for i, (p, f) in enumerate(zip(plans, fs)):
                per_eps_ev[s][i][0].record(stream)
                p.exec(c, f, stream=stream)
                per_eps_ev[s][i][1].record(stream)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    eps_ms = [[per_eps_ev[s][i][0].elapsed_time(per_eps_ev[s][i][1]) for s in range(args.steps)]
              for i in range(len(plans))]
    stats = [p.stage_stats() for p in plans]
    for p in plans:
        p.set_timing(False)
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    coeffs_per_step = len(plans) * N * nrhs
    value = world * coeffs_per_step * args.steps / (total_ms / 1000.0)

    # dominant kernel: the FFT passes (FP64, bound by the FP64 pipe, not HBM)
    fft_ms = sum(st["fft"]["ms"] for st in stats)
    fft_flops = sum(st["fft"]["flops"] for st in stats)
    fft_launches = sum(st["fft"]["launches"] for st in stats)
    fft_bytes = sum(st["fft"]["bytes"] for st in stats)
    achieved = fft_flops / (fft_ms / 1000.0) / 1e9 if fft_ms > 0 else 0.0
    launches = sum(st[k]["launches"] for st in stats for k in st)
    stage_ms = {k: round(sum(st[k]["ms"] for st in stats) / args.steps, 3) for k in stats[0]}

    # end to end: host arrays in and out through the C ABI, copies inside the timed region
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(1, min(args.steps, 2))
    c_pin = torch.from_numpy(c_host).pin_memory()
    f_pin = torch.empty((nrhs, N), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for p in plans:
            p.exec_host(c_pin.numpy(), out=f_pin.numpy())
    e2e_s = time.perf_counter() - t0
    e2e_value = world * coeffs_per_step * e2e_steps / e2e_s

    fp32 = all(p.info["precision"] == 2 for p in plans)
    pass_gbs = fft_bytes / (fft_ms / 1000.0) / 1e9 if fft_ms > 0 else None
    if fp32:
        # FP32 stages are memory-bound: report the FFT passes against HBM bandwidth
        peak, src = hbm_peak()
        roofline = {"bound": "hbm", "achieved": pass_gbs, "peak": peak, "unit": "GB/s",
                    "frac": (pass_gbs or 0.0) / peak, "traffic": None, "peak_source": src,
                    "kernel": "k_fft_pass (FP32 Stockham passes, forward + inverse)",
                    "bytes_model": "each pass reads and writes every point once (16 B per complex float)",
                    "launches": fft_launches}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                    "frac": achieved / FP64_PEAK_GFLOPS,
                    "traffic": FFT_TRAFFIC_RATIO * fft_bytes / fft_launches if fft_launches else None,
                    "traffic_unit": "DRAM bytes per launch (ncu ratio x algorithmic bytes)",
                    "frac_of_measured_fp64": achieved / FP64_MEASURED_GFLOPS, "hbm_gbs_of_passes": pass_gbs,
                    "kernel": "k_fft_pass (FP64 Stockham passes, forward + inverse)",
                    "flops_model": "5 F log2 F per column transform", "launches": fft_launches,
                    "peak_source": "nominal FP64 from unit counts and clock (152 SM x 4 flop/clk x 2.07 GHz)"}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "coeffs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
        "config": {"workload": "dht0_N%d_eps%s_nrhs%d_plain" % (N, "+".join(args.eps.split(",")), nrhs),
                   "N": N, "eps": eps_list, "nrhs": nrhs,
                   "form": "plain per-request " + ("FP32 stages (eps >= 1e-5)" if fp32 else "FP64"),
                   "l2": "flushed between timed steps (256 MB write)", "coefficients": "N(0,1) seeded"},
        "per_eps": {str(e): {"ms": statistics.mean(m), "coeffs_per_s": N * nrhs / (statistics.mean(m) / 1000.0),
                             "p50_ms": statistics.median(m), "p99_ms": max(m)}
                    for e, m in zip(eps_list, eps_ms)},
        "stage_ms_per_step": stage_ms,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "coeffs/s", "h2d_bytes_per_step": len(plans) * N * nrhs * 8,
                "d2h_bytes_per_step": len(plans) * N * nrhs * 8, "steps": e2e_steps},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "wall_s_timed": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(N, args.cpu_rows, seed_for(4, 99))
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
