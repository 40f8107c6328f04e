#!/usr/bin/env python
"""Benchmark: DHT-0 coefficients/s at N = 2^20, eps in {1e-15, 1e-8}, FP64, one GB300.

One step = one discrete Hankel transform of order 0 (Section 6, Eq. 25) at eps = 1e-15 plus
one at eps = 1e-8, each over a batch of ``--nrhs`` seeded standard-normal coefficient vectors
(the paper's Gaussian experiments): the served/batched form, every stage FP64 (the AUTO
precision below eps = 1e-5). value = coefficients transformed / device time with the inputs
resident. The line also carries the plain form (one vector per execution, FP64) measured the
same way, the opt-in mixed-precision batched form (double-float and FP32 terms) as a separate
key with its own error against the oracle, and both FP64 forms driven through the library's
request loop with host arrays: throughput when all requests arrive at once (e2e) and p50/p99
latency under Poisson arrivals.

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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from hankel_inputs import coefficients, sample_rows, seed_for  # noqa: E402

FP64_PEAK_GFLOPS = 152 * 4 * 2.07  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz = 1258 GFLOP/s
HBM_FALLBACK_GBS = 6800.0          # used only when MEASURED_PEAKS.json is absent
FP64_MEASURED_GFLOPS = 1004.0      # DFMA microbenchmark on this part (2 x 502 G instructions/s)
# DRAM bytes per algorithmic byte of an FFT pass launch of FP64 transforms, from an ncu capture of
# three passes on the tensor cores over 16 x 2^21 points (two radix-32 passes by twiddle group, one
# stride-1 radix-64 pass): 3328.8 MB of DRAM reads + writes against 3 x 1073.7 MB algorithmic.
FFT_TRAFFIC_RATIO = (537.629 + 494.579 + 563.824 + 496.177 + 731.730 + 504.892) / (3 * 1073.742)
# Executed fp16 MMA flops per complex point of a tensor-core radix-32 pass: 34 digit-plane products
# of 128 x 64 x 16 in each of 4 K steps per tile of 4096 points.
TC_MMA_FLOPS_PER_POINT = (2 * 128 * 16 * 64 * 34 * 4) / 4096.0
# The double-float transforms are bound by the FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz =
# 40.3 T instructions/s. Their radix-2 butterfly (two double-float dot products of 16 FP32
# instructions each, four sums of 8) takes 64 FP32 instructions for the 10 flops of the
# 5 F log2 F model, so the pipe bounds the model rate at 40.3 T / 6.4.
FP32_ISSUE_PEAK = 152 * 128 * 2.07e9
DF64_INSTR_PER_FLOP = 6.4
DF64_PEAK_GFLOPS = FP32_ISSUE_PEAK / DF64_INSTR_PER_FLOP / 1e9
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
    ap.add_argument("--nrhs", type=int, default=16, help="vectors per batched execution (served form)")
    ap.add_argument("--requests", type=int, default=0,
                    help="single-vector requests per serving run (0: nrhs per eps, the batched step's vectors)")
    ap.add_argument("--rate", type=float, default=0.0, help="Poisson request rate (0: 70%% of plain capacity)")
    ap.add_argument("--eps", default="1e-15,1e-8")
    ap.add_argument("--cpu-rows", type=int, default=4096, help="oracle rows per sample (about 10 s on 16 cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="dht", choices=["dht", "mix"], help="mix: the serving-mix workload")
    ap.add_argument("--quick", action="store_true", help="batched form only (no plain form, serving runs or CPU leg)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the opt-in mixed-precision batched form")
    ap.add_argument("--fp32-eps", type=float, default=1e-4,
                    help="tolerance of the FP32-stage batched form reported beside the value (0: skip)")
    ap.add_argument("--mix-requests", type=int, default=1000, help="requests per arrival rate")
    ap.add_argument("--mix-rates", default="100,1000,10000", help="Poisson arrivals per second, one run each")
    ap.add_argument("--mix-nmin", type=int, default=10)
    ap.add_argument("--mix-nmax", type=int, default=20)
    ap.add_argument("--mix-vmax", type=int, default=64)
    ap.add_argument("--clocks-csv", default=None,
                    help="keep the nvidia-smi samples of the timed region in this file (default: a temporary file)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    def __init__(self, index, path=None):
        self.index = index
        self.proc = None
        self.keep = path is not None
        if path is None:
            fd, path = tempfile.mkstemp(prefix="bench_clocks_%d_" % index, suffix=".csv")
            os.close(fd)
        self.path = path

    def __enter__(self):
        try:
            if os.path.dirname(self.path):
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
        if not self.keep:
            os.remove(self.path)
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
    rows = base_rows(N, rows_count, seed)
    t0 = time.perf_counter()
    f = oracle.transform("dht", 0, N, c, rows=rows)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    # one output row costs N J-evaluations; a full transform is N rows, so coefficients/s = rows/s
    return {"value": len(rows) / dt, "unit": "coeffs/s", "cores": cores, "kind": "oracle",
            "sample": "%d of %d rows of one DHT-0 at N=%d (direct O(N^2) FP64 Kahan sum; rows/s = "
                      "coefficients/s of a full transform)" % (len(rows), N, N),
            "seconds": dt, "f": np.asarray(f).reshape(-1)}


def base_rows(N, rows_count, seed):
    """Rows (0-based) the CPU baseline evaluates."""
    return sample_rows(N, rows_count, seed + 1)


def workload_config(args):
    """The workload both arms report: DHT-0 at N, every eps of --eps, batches of --nrhs vectors."""
    B = args.nrhs
    return {"workload": "dht0_N%d_eps%s_batch%d" % (args.N, "+".join(args.eps.split(",")), B),
            "N": args.N, "eps": [float(e) for e in args.eps.split(",")], "batch": B,
            "form": "served/batched: %d vectors per execution per plan, every stage FP64 (AUTO precision "
                    "below eps = 1e-5)" % B,
            "l2": "flushed between timed steps (256 MB write)", "coefficients": "N(0,1) seeded"}


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
        r.pop("f")
        if step >= args.warmup:
            times.append(r["seconds"])
            rows_total += args.cpu_rows
    # the oracle's cost does not depend on eps; one step covers both eps values of the workload
    value = rows_total / sum(times)
    ms_per_step = 1000.0 * len(eps) * N * args.nrhs / value  # the same step as the GPU arm: every eps, a batch
    cores = len(os.sched_getaffinity(0))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "coeffs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args), sample_rows_per_step=args.cpu_rows),
        "cpu_baseline": {"value": value, "unit": "coeffs/s", "cores": cores, "kind": "oracle",
                         "sample": "%d seeded rows per step of a DHT-0 at N=%d" % (args.cpu_rows, N)},
        "e2e": {"value": value, "unit": "coeffs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def aggregate(world, coeffs_per_step, steps, total_ms, device):
    """Whole-job throughput of `world` replicas: the slowest rank's summed step time over
    every rank's coefficients. Returns (value, max_total_ms)."""
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * coeffs_per_step * steps / (total_ms / 1000.0), total_ms


def timed_steps(plans, c, fs, stream, steps, warmup, flush, timing, concurrent=False):
    """Warm up, then time `steps` steps (each: every plan once) with CUDA events on `stream`.

    L2 is flushed between steps, outside the step events. With `concurrent`, each plan runs on
    a stream of its own, forked from and joined back to `stream` (as the request loop runs
    different plans); otherwise the plans run one after another on `stream`. Returns per-step
    ms, per-plan ms lists and (when timing) the plans' stage statistics."""
    import torch

    pstreams = [torch.cuda.Stream() for _ in plans] if concurrent else [stream for _ in plans]

    def one_step(pev=None):
        if concurrent:
            fork = torch.cuda.Event()
            fork.record(stream)
        joins = []
        for i, (p, f) in enumerate(zip(plans, fs)):
            ps = pstreams[i]
            if concurrent:
                ps.wait_event(fork)
            if pev is not None:
                pev[i][0].record(ps)
            p.exec(c, f, stream=ps)
            if pev is not None:
                pev[i][1].record(ps)
            if concurrent:
                j = torch.cuda.Event()
                j.record(ps)
                joins.append(j)
        for j in joins:
            stream.wait_event(j)

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    if timing:
        for p in plans:
            p.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    pev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in plans]
           for _ in range(steps)]
    torch.cuda.synchronize()
    for s in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[s][0].record(stream)
        one_step(pev[s])
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    plan_ms = [[pev[s][i][0].elapsed_time(pev[s][i][1]) for s in range(steps)] for i in range(len(plans))]
    stats = [p.stage_stats() for p in plans] if timing else None
    if timing:
        for p in plans:
            p.set_timing(False)
    return step_ms, plan_ms, stats


def pinned_like(a):
    """A page-locked host array with a's shape and contents (float64)."""
    import torch

    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    out = t.numpy()
    out[...] = a
    return out


def serve_stream(hk, server_kw, requests, rate, seed, rounds=1):
    """Feed `requests` [(eps, c)] to a server with Poisson arrivals at `rate` per second
    (rate <= 0: all at once), `rounds` times. Returns (coefficients/s over the summed makespans,
    latencies in ms of every request)."""
    srv = hk.Server(**server_kw)
    outs = [pinned_like(c) for _, c in requests]
    # warm-up (untimed): two all-at-once rounds build the plans and (a plan's first run is not
    # captured) capture the graphs of the batch sizes an all-at-once arrival forms; then single
    # requests for the sizes of spread-out arrivals
    for _ in range(2):
        warm = [srv.submit("dht", 0, c.shape[-1], eps, c, f)[0] for (eps, c), f in zip(requests, outs)]
        for t in warm:
            srv.wait(t)
    for _ in range(2):
        for (eps, c), f in zip(requests[:2], outs):
            t, _ = srv.submit("dht", 0, c.shape[-1], eps, c, f)
            srv.wait(t)
    rng = np.random.default_rng(seed)
    lat, makespan = [], 0.0
    for _ in range(rounds):
        gaps = rng.exponential(1.0 / rate, size=len(requests)) if rate > 0 else np.zeros(len(requests))
        t0 = time.perf_counter()
        due = t0
        tickets = []
        for (eps, c), gap in zip(requests, gaps):
            due += gap
            while time.perf_counter() < due:
                time.sleep(min(0.001, max(0.0, due - time.perf_counter())))
            tickets.append(srv.submit("dht", 0, c.shape[-1], eps, c, outs[len(tickets)])[0])
        lat += [srv.wait(t) for t in tickets]
        makespan += time.perf_counter() - t0
    coeffs = rounds * sum(c.size for _, c in requests)
    srv.close()
    return coeffs / makespan, lat


def pct(values, q):
    return float(np.percentile(np.asarray(values), q)) if values else None


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    import paper_1501_01652_gb300 as hk

    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, B = args.N, args.nrhs
    eps_list = [float(e) for e in args.eps.split(",")]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    # plain form: one vector per execution, every stage FP64
    plain_cps, p_step, p_plan = None, [float("nan")], [[float("nan")] for _ in eps_list]
    if not args.quick:
        c1_host = coefficients("normal", N, 1, seed_for(4, rank))
        c1 = torch.from_numpy(c1_host).to(dev)
        plain = [hk.Plan("dht", 0, N, e, precision="fp64") for e in eps_list]
        f1 = [torch.empty((1, N), dtype=torch.float64, device=dev) for _ in plain]
        p_step, p_plan, _ = timed_steps(plain, c1, f1, stream, max(1, args.steps), 1, flush, False)
        plain_cps = len(plain) * N * len(p_step) / (sum(p_step) / 1000.0)
        for p in plain:
            p.destroy()

    # served form: batches of B vectors per plan, every stage FP64 (AUTO below eps = 1e-5)
    cB_host = coefficients("normal", N, B, seed_for(4, 100 + rank))
    cB = torch.from_numpy(cB_host).to(dev)
    plans = [hk.Plan("dht", 0, N, e, max_nrhs=B) for e in eps_list]
    fs = [torch.empty((B, N), dtype=torch.float64, device=dev) for _ in plans]
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local, args.clocks_csv) as clocks:
        wall0 = time.perf_counter()
        step_ms, plan_ms, _ = timed_steps(plans, cB, fs, stream, args.steps, args.warmup, flush, False)
        wall = time.perf_counter() - wall0
    # the stage split from further steps with per-stage events (outside the timed region)
    ev_step_ms, _, stats = timed_steps(plans, cB, fs, stream, args.steps, 0, flush, True)
    if world > 1:
        torch.distributed.barrier()
    coeffs_per_step = len(plans) * N * B
    value, total_ms = aggregate(world, coeffs_per_step, args.steps, sum(step_ms), dev)

    # launches of the stage-timed steps, as many as the timed region's
    launches = sum(st[k]["launches"] for st in stats for k in st)
    # the autotuner's launch splits of the timed plans, with its own measurements (default vs chosen)
    tuned = [dict(sh, plan_eps=e) for p, e in zip(plans, eps_list) for sh in p.fft_shapes()]
    measured = [t for t in tuned if t["ms_default"] > 0]
    autotune = {"shapes": tuned,
                "chosen_over_default": (sum(t["ms_chosen"] for t in measured) / sum(t["ms_default"] for t in measured))
                if measured else None,
                "note": "per (precision, log2 length, column bucket): the built-in split and the chosen one, timed "
                        "at plan creation on the plan's workspace (ms of one launch sequence)"}
    stage_ms = {k: round(sum(st[k]["ms"] for st in stats) / args.steps, 3) for k in stats[0]}
    roofline = fft_roofline(stats, args.steps)
    hbm_stages = stage_hbm(stats, args.steps)
    precs = [p.info["precision"] for p in plans]
    terms = term_counts(plans)
    dtype = dtype_of(precs, terms)
    # accuracy of the timed plans on the CPU baseline's vector and rows (checked by the oracle
    # there, outside every timed region)
    err_c = coefficients("normal", N, 1, seed_for(4, 99))
    want_err = world == 1 and not args.no_cpu_baseline and not args.quick
    ce = torch.from_numpy(err_c).to(dev)
    f_err = [p.exec(ce).cpu().numpy()[0] for p in plans] if want_err else []
    tc_pass = tensor_pass_roofline(hk, plans, args.steps)
    for p in plans:
        p.destroy()

    # the opt-in mixed-precision batched form (double-float plans at 1e-8, double-float and FP32
    # low-rank terms): reported beside the FP64 value, never as it
    mixed = None
    if not args.no_mixed:
        mplans = [hk.Plan("dht", 0, N, e, max_nrhs=B, precision="mixed") for e in eps_list]
        m_step, m_plan, _ = timed_steps(mplans, cB, fs, stream, args.steps, args.warmup, flush, False)
        _, _, m_stats = timed_steps(mplans, cB, fs, stream, 1, 0, flush, True)
        m_value = coeffs_per_step * len(m_step) / (sum(m_step) / 1000.0)
        m_terms = term_counts(mplans)
        m_err = [p.exec(ce).cpu().numpy()[0] for p in mplans] if want_err else []
        mixed = {"value": m_value, "unit": "coeffs/s", "ms_per_step": sum(m_step) / len(m_step),
                 "dtype": dtype_of([p.info["precision"] for p in mplans], m_terms),
                 "over_fp64_value": m_value / value,
                 "per_eps_ms": {str(e): statistics.mean(m) for e, m in zip(eps_list, m_plan)},
                 "term_precision": {"fp64": m_terms[0], "df64": m_terms[1], "fp32": m_terms[2]},
                 "stage_ms_per_step": {k: round(sum(st[k]["ms"] for st in m_stats), 3) for k in m_stats[0]},
                 "form": "precision='mixed': narrower than FP64 below eps = 1e-5 by explicit opt-in"}
        for p in mplans:
            p.destroy()

    # the default policy's FP32-stage class (eps >= 1e-5): one batched plan, its transforms against
    # the measured HBM copy rate; reported beside the FP64 value, never as it
    fp32 = None
    if args.fp32_eps > 0:
        p32 = [hk.Plan("dht", 0, N, args.fp32_eps, max_nrhs=B)]
        f32 = [fs[0]]
        s_step, _, _ = timed_steps(p32, cB, f32, stream, args.steps, args.warmup, flush, False)
        _, _, s_stats = timed_steps(p32, cB, f32, stream, args.steps, 0, flush, True)
        s_err = p32[0].exec(ce).cpu().numpy()[0] if want_err else None
        s_roof = fft_roofline(s_stats, args.steps)
        fp32 = {"eps": args.fp32_eps, "dtype": dtype_of([p32[0].info["precision"]], term_counts(p32)),
                "ms_per_step": sum(s_step) / len(s_step),
                "coeffs_per_s": N * B * len(s_step) / (sum(s_step) / 1000.0),
                "stage_ms_per_step": {k: round(sum(st[k]["ms"] for st in s_stats) / args.steps, 3)
                                      for k in s_stats[0]},
                "roofline": s_roof,
                "form": "default policy at eps >= 1e-5: FP32 stages, %d vectors per execution" % B}
        p32[0].destroy()
    del fs

    # request streams through the library's server: end to end with host arrays
    reqs = []
    nreq = args.requests if args.requests > 0 else B * len(eps_list)
    for i in range(nreq):
        e = eps_list[i % len(eps_list)]
        reqs.append((e, pinned_like(coefficients("normal", N, 1, seed_for(4, 200 + i))[0])))
    # batches of at most 2 vectors (spread-out arrivals) run on plans built for 2; one batch of a plan
    # at a time (the requests of this stream all share two plans: a second context would run a
    # plan's batches side by side, each slower, where in turn and packed they finish sooner)
    served_kw = dict(streams=4, max_batch=B, use_graphs=True, precision="auto", small_batch=2, contexts_per_plan=1)
    plain_kw = dict(streams=1, max_batch=1, use_graphs=False, precision="fp64", pack=False)
    if args.quick:
        served_e2e = plain_e2e = served_cps_p = plain_cps_p = rate = None
        served_sat_lat = plain_sat_lat = served_lat = plain_lat = []
    else:
        served_e2e, served_sat_lat = serve_stream(hk, served_kw, reqs, 0.0, 1, rounds=args.steps)
        plain_e2e, plain_sat_lat = serve_stream(hk, plain_kw, reqs, 0.0, 1, rounds=args.steps)
        rate = args.rate if args.rate > 0 else 0.7 * plain_e2e / N  # 70 % of the plain form's capacity
        # four rounds of the 32 arrivals: 128 latencies per form
        served_cps_p, served_lat = serve_stream(hk, served_kw, reqs, rate, 2, rounds=4)
        plain_cps_p, plain_lat = serve_stream(hk, plain_kw, reqs, rate, 2, rounds=4)

    term_split = {"fp64": terms[0], "df64": terms[1], "fp32": terms[2],
                  "unit": "far-field transforms per right-hand side, summed over blocks and plans"}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "coeffs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": workload_config(args),
        "per_eps": {str(e): {"batch_ms": statistics.mean(m),
                             "coeffs_per_s": N * B / (statistics.mean(m) / 1000.0),
                             "plain_ms": statistics.mean(pm) if plain_cps else None,
                             "plain_coeffs_per_s": N / (statistics.mean(pm) / 1000.0) if plain_cps else None,
                             "mixed_batch_ms": mixed["per_eps_ms"][str(e)] if mixed else None}
                    for e, m, pm in zip(eps_list, plan_ms, p_plan)},
        "plain_fp64": {"coeffs_per_s": plain_cps, "ms_per_step": (sum(p_step) / len(p_step)) if plain_cps else None,
                       "form": "one vector per execution, every stage FP64"},
        "served_over_plain": value / plain_cps if plain_cps else None,
        "mixed_precision": mixed,
        "fp32_stages": fp32,
        "stage_ms_per_step": stage_ms,
        "stage_steps_ms": sum(ev_step_ms) / len(ev_step_ms),
        "term_precision": term_split,
        "roofline": roofline,
        "hbm_stages": hbm_stages,
        "tensor_core_pass": tc_pass,
        "fft_autotune": autotune,
        "e2e": {"value": served_e2e, "unit": "coeffs/s", "h2d_bytes_per_step": coeffs_per_step * 8,
                "d2h_bytes_per_step": coeffs_per_step * 8,
                "form": "hankel_server (FP64 plans), %d single-vector requests (%d per eps) submitted at once, "
                        "page-locked host arrays (inputs and outputs); %d such rounds after 2 untimed ones"
                        % (len(reqs), len(reqs) // len(eps_list), args.steps),
                "plain_value": plain_e2e},
        "latency_ms": {"rate_per_s": rate, "requests": 4 * len(reqs) if rate else len(reqs),
                       "served": {"p50": pct(served_lat, 50), "p99": pct(served_lat, 99),
                                  "coeffs_per_s": served_cps_p},
                       "plain": {"p50": pct(plain_lat, 50), "p99": pct(plain_lat, 99),
                                 "coeffs_per_s": plain_cps_p},
                       "saturated": {"served_p50": pct(served_sat_lat, 50), "served_p99": pct(served_sat_lat, 99),
                                     "plain_p50": pct(plain_sat_lat, 50), "plain_p99": pct(plain_sat_lat, 99)}},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "wall_s_timed": wall,
    }
    if want_err:
        base = cpu_baseline(N, args.cpu_rows, seed_for(4, 99))
        ref = base.pop("f")
        line["cpu_baseline"] = base
        # max over the sampled rows of |f - f_oracle| / (eps sum|c|); the parity bar is 10
        l1 = float(np.abs(err_c).sum())
        rows = base_rows(N, args.cpu_rows, seed_for(4, 99))
        line["error_vs_oracle"] = {str(e): float(np.max(np.abs(f[rows] - ref)) / (e * l1))
                                   for e, f in zip(eps_list, f_err)}
        if fp32 is not None and s_err is not None:
            fp32["error_vs_oracle"] = {str(args.fp32_eps): float(np.max(np.abs(s_err[rows] - ref)) /
                                                                 (args.fp32_eps * l1))}
        if mixed:
            mixed["error_vs_oracle"] = {str(e): float(np.max(np.abs(f[rows] - ref)) / (e * l1))
                                        for e, f in zip(eps_list, m_err)}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def tensor_pass_roofline(hk, plans, steps):
    """The longest transform the plans run with tensor-core passes, timed alone (CUDA events, outside
    the timed region) in its tuned split and in the built-in FP64 one; the executed fp16 MMA rate of
    its radix-32 passes against the measured bf16 peak (the fp16 rate)."""
    best = None
    for p in plans:
        for sh in p.fft_shapes():
            if any(sh["tensor_passes"]) and (best is None or (sh["log2_len"], sh["col_bucket"]) >
                                              (best["log2_len"], best["col_bucket"])):
                best = sh
    if best is None:
        return None
    logF, rad = best["log2_len"], best["radices"]
    mask = sum(1 << i for i, t in enumerate(best["tensor_passes"]) if t)
    ncols = max(1, min(1 << best["col_bucket"], (1 << 25) >> logF))
    err, ms = hk.debug_fft_compare(logF, ncols, rad, mask)
    # the same length on the FP64 pipe in the library's built-in split (the fewest passes of radix
    # up to 2^8, as equal as possible)
    npass = (logF + 7) // 8
    while npass > 1 and logF // npass < 5:
        npass -= 1
    builtin = [logF // npass + (1 if i < logF % npass else 0) for i in range(npass)]
    try:
        _, ms64 = hk.debug_fft_compare(logF, ncols, builtin, 0)
    except RuntimeError:
        ms64 = None
    points = ncols * (1 << logF)
    ntc = sum(1 for t in best["tensor_passes"] if t)
    peak = bf16_peak()
    mma = TC_MMA_FLOPS_PER_POINT * points * ntc / (ms / 1000.0) / 1e12
    return {"log2_len": logF, "ncols": ncols, "radices": rad, "tensor_passes": best["tensor_passes"],
            "ms": ms, "ms_fp64_pipe": ms64, "fp64_pipe_radices": builtin,
            "speedup_over_fp64_pipe": (ms64 / ms) if ms64 else None,
            "max_rel_diff_vs_fp64_pipe": err,
            "fp64_equiv_gflops": 5.0 * points * logF / (ms / 1000.0) / 1e9,
            "mma_tflops": mma, "bound": "tensor", "peak": peak, "unit": "TFLOP/s", "frac": mma / peak,
            "note": "executed fp16 digit-product MMA flops (radix-32 count per pass) over the whole transform's "
                    "time; the passes are issue-bound on the integer pipe (profiles/k_fft_pass_tc_*)"}


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def term_counts(plans):
    """Far-field transforms per right-hand side in FP64, double-float and FP32, over all plans."""
    terms = [0, 0, 0]
    for p in plans:
        for b in p.blocks():
            for i in range(3):
                terms[i] += b["terms"][i]
    return terms


def dtype_of(precs, terms):
    kinds = ["f64" if (1 in precs or terms[0]) else None, "df64" if (3 in precs or terms[1]) else None,
             "f32" if (2 in precs or terms[2]) else None]
    return "+".join(k for k in kinds if k)


def stage_hbm(stats, steps):
    """The segment sums (`k_seg_mac`) and row sums (`k_out`) against both of their bounds: the
    measured HBM copy rate for their algorithmic bytes, and the FP64 pipe for their complex
    multiply-adds (4 DFMA per point and segment, 2 per column and row), which binds on this part."""
    peak, src = hbm_peak()
    out = {"peak": peak, "unit": "GB/s", "peak_source": src,
           "bytes_model": "every operand read once and every result written once",
           "flops_model": "segment sums 8 flop per point and segment, row sums 4 flop per column and row",
           "fp64_peak_gflops": FP64_PEAK_GFLOPS, "fp64_measured_gflops": FP64_MEASURED_GFLOPS}
    for k, kern in (("pointwise", "k_seg_mac"), ("out", "k_out")):
        ms = sum(st[k]["ms"] for st in stats)
        by = sum(st[k]["bytes"] for st in stats)
        fl = sum(st[k]["flops"] for st in stats)
        gbs = by / (ms / 1000.0) / 1e9 if ms > 0 else None
        gfl = fl / (ms / 1000.0) / 1e9 if ms > 0 else None
        out[k] = {"kernel": kern, "ms_per_step": ms / steps, "gbytes_per_step": by / steps / 1e9,
                  "launches": sum(st[k]["launches"] for st in stats) // steps, "achieved": gbs,
                  "frac": (gbs / peak) if gbs else None, "gflops": gfl,
                  "frac_of_fp64_peak": (gfl / FP64_PEAK_GFLOPS) if gfl else None,
                  "frac_of_measured_fp64": (gfl / FP64_MEASURED_GFLOPS) if gfl else None}
    return out


def fft_roofline(stats, steps):
    """Roofline entry of the transform class (FP64, double-float or FP32 passes) that takes the
    most time, with the other classes under "others"."""

    def fft_entry(k2):
        ms2 = sum(st[k2]["ms"] for st in stats)
        fl = sum(st[k2]["flops"] for st in stats)
        nl = sum(st[k2]["launches"] for st in stats)
        by = sum(st[k2]["bytes"] for st in stats)
        ach = fl / (ms2 / 1000.0) / 1e9 if ms2 > 0 else 0.0
        gbs = by / (ms2 / 1000.0) / 1e9 if ms2 > 0 else None
        common = {"fft_ms_per_step": ms2 / steps, "launches": nl, "hbm_gbs_of_passes": gbs,
                  "flops_model": "5 F log2 F per column transform, plus 6 F per spectrum product folded "
                                 "into an inverse transform"}
        if k2 == "fft":
            e = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                 "frac": ach / FP64_PEAK_GFLOPS,
                 "traffic": FFT_TRAFFIC_RATIO * by / nl if nl else None,
                 "traffic_unit": "DRAM bytes per launch (ncu ratio of the tensor-core pass x algorithmic bytes)",
                 "frac_of_measured_fp64": ach / FP64_MEASURED_GFLOPS,
                 "kernel": "FP64-accuracy transforms: k_fft_pass_tc (radix-32/64 passes on the tensor cores) and "
                           "k_fft_pass_reg / k_fft_small<double2> (FP64 pipe), forward + inverse",
                 "peak_source": "nominal FP64 from unit counts and clock (152 SM x 4 flop/clk x 2.07 GHz): the "
                                "pipe these transforms would run on without the tensor cores; a frac_of_measured_fp64 "
                                "above 1 is the tensor-core passes beating that roofline"}
        elif k2 == "fft_df64":
            e = {"bound": "alu", "achieved": ach, "peak": DF64_PEAK_GFLOPS, "unit": "GFLOP/s",
                 "frac": ach / DF64_PEAK_GFLOPS, "traffic": None,
                 "kernel": "k_fft_pass_reg / k_fft_small<df64c> (double-float transforms, forward + inverse)",
                 "peak_source": "FP32 pipe (152 SM x 128 lanes x 2.07 GHz) / 6.4 FP32 instructions per "
                                "double-float flop of the butterfly"}
        else:
            peak, src = hbm_peak()
            e = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": (gbs or 0.0) / peak,
                 "traffic": None, "peak_source": src,
                 "kernel": "k_fft_pass_reg / k_fft_small<float2> (FP32 transforms, forward + inverse)",
                 "bytes_model": "each pass reads and writes every point once (8 B read + 8 B written per "
                                "complex float point)",
                 "gflops_5FlogF": ach}
        e.update(common)
        return e

    classes = [k2 for k2 in ("fft", "fft_df64", "fft_fp32") if sum(st[k2]["ms"] for st in stats) > 0]
    dominant = max(classes, key=lambda k2: sum(st[k2]["ms"] for st in stats)) if classes else "fft"
    roofline = fft_entry(dominant)
    names = {"fft": "fp64_transforms", "fft_df64": "df64_transforms", "fft_fp32": "fp32_transforms"}
    roofline["others"] = {names[k2]: fft_entry(k2) for k2 in classes if k2 != dominant}
    return roofline


MIX_TASKS = [("schlomilch", 0), ("schlomilch", 1), ("fourier_bessel", 0), ("dht", 0)]
MIX_EPS = [1e-15, 1e-8, 1e-4]


def mix_requests(args):
    """Seeded serving mix: task uniform over MIX_TASKS, N = 2^k with k uniform in
    [mix_nmin, mix_nmax] (log-uniform N), eps uniform over MIX_EPS, 1..mix_vmax vectors. A request's
    coefficients are the first vectors of a seeded uniform[-1, 1] pool of its N (one pool of mix_vmax
    vectors per N keeps the host memory of a thousand requests bounded)."""
    rng = np.random.default_rng(seed_for(5, 0))
    pools = {}
    reqs = []
    for i in range(args.mix_requests):
        task, nu = MIX_TASKS[rng.integers(len(MIX_TASKS))]
        N = 1 << int(rng.integers(args.mix_nmin, args.mix_nmax + 1))
        eps = MIX_EPS[rng.integers(len(MIX_EPS))]
        nv = int(rng.integers(1, args.mix_vmax + 1))
        if N not in pools:
            pools[N] = coefficients("uniform", N, args.mix_vmax, seed_for(5, 1 + len(pools)))
        reqs.append((task, nu, N, eps, pools[N][:nv]))
    return reqs


def warm_plans(srv, reqs):
    """Build every plan key of the stream once (one one-vector request each), outside the timing."""
    seen = set()
    for task, nu, N, eps, c in reqs:
        if (task, nu, N, eps) not in seen:
            seen.add((task, nu, N, eps))
            t, _ = srv.submit(task, nu, N, eps, c[:1])
            srv.wait(t)
    return len(seen)


def run_mix_stream(srv, reqs, rate, seed):
    """Submit reqs with Poisson arrivals at `rate` per second; every request's latency is its
    submission-to-completion time. Returns throughput over the makespan and p50/p99 latency."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=len(reqs))
    # output arrays: one pool per N (requests in flight at once may share one; only the timing is read)
    outs = {}
    vmax = max(c.shape[0] for *_, c in reqs)
    for *_, c in reqs:
        if c.shape[1] not in outs:
            outs[c.shape[1]] = np.empty((vmax, c.shape[1]))
    before = srv.stats()
    t0 = time.perf_counter()
    due = t0
    tickets = []
    for (task, nu, N, eps, c), gap in zip(reqs, gaps):
        due += gap
        while time.perf_counter() < due:
            time.sleep(min(0.0005, max(0.0, due - time.perf_counter())))
        tickets.append(srv.submit(task, nu, N, eps, c, outs[N][:c.shape[0]])[0])
    lat = [srv.wait(t) for t in tickets]
    makespan = time.perf_counter() - t0
    st = srv.stats()
    coeffs = sum(c.size for *_, c in reqs)
    return {"rate_per_s": rate, "requests": len(reqs), "coeffs_per_s": coeffs / makespan, "p50_ms": pct(lat, 50),
            "p99_ms": pct(lat, 99), "max_ms": max(lat), "makespan_s": makespan,
            "batches": st["batches"] - before["batches"], "contexts_added": st["contexts_added"],
            "plans_built": st["plans_built"], "plans_evicted": st["plans_evicted"],
            "graphs": st["graphs_captured"], "device_bytes": st["device_bytes"]}


def run_mix(args):
    """Serving mix through the request loop: served (packed batches on 4 streams, up to two batches
    of one plan in flight, CUDA graphs, AUTO precision: FP64 below eps = 1e-5, FP32 stages above)
    against plain (one request at a time, every stage FP64), the same arrival streams, at each rate
    of --mix-rates."""
    import torch

    import paper_1501_01652_gb300 as hk

    torch.cuda.set_device(0)
    reqs = mix_requests(args)
    rates = [float(r) for r in args.mix_rates.split(",")]
    forms = {"served": dict(streams=4, max_batch=64, use_graphs=True, precision="auto", contexts_per_plan=2),
             "plain_fp64": dict(streams=1, max_batch=64, use_graphs=False, precision="fp64", pack=False,
                                contexts_per_plan=1)}
    out = {}
    for name, kw in forms.items():
        srv = hk.Server(memory_cap=120 << 30, **kw)
        t0 = time.perf_counter()
        keys = warm_plans(srv, reqs)
        warm_s = time.perf_counter() - t0
        out[name] = {"plan_keys": keys, "plan_warmup_s": warm_s,
                     "per_rate": [run_mix_stream(srv, reqs, rate, 3 + i) for i, rate in enumerate(rates)]}
        srv.close()
    per_rate = []
    for i, rate in enumerate(rates):
        sv, pl = out["served"]["per_rate"][i], out["plain_fp64"]["per_rate"][i]
        per_rate.append({"rate_per_s": rate, "served_coeffs_per_s": sv["coeffs_per_s"],
                         "plain_coeffs_per_s": pl["coeffs_per_s"],
                         "served_over_plain": sv["coeffs_per_s"] / pl["coeffs_per_s"],
                         "served_p50_ms": sv["p50_ms"], "served_p99_ms": sv["p99_ms"],
                         "plain_p50_ms": pl["p50_ms"], "plain_p99_ms": pl["p99_ms"],
                         "p99_plain_over_served": pl["p99_ms"] / sv["p99_ms"]})
    line = {"metric": "serving mix coeffs/s and p50/p99 ms, served vs plain FP64",
            "value": per_rate[len(per_rate) // 2]["served_coeffs_per_s"], "unit": "coeffs/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "serving_mix", "requests_per_rate": len(reqs), "rates_per_s": rates,
                       "N": "2^%d..2^%d log-uniform" % (args.mix_nmin, args.mix_nmax),
                       "vectors_per_request": "1..%d" % args.mix_vmax, "eps": MIX_EPS,
                       "tasks": ["%s-%d" % t for t in MIX_TASKS], "memory_cap_gib": 120},
            "per_rate": per_rate, "detail": out}
    print(json.dumps(line))


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "mix":
        run_mix(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
