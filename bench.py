#!/usr/bin/env python
"""Benchmark: dense univariate evaluation at 2^24 points.

Workload (one step): polynomials with k = 1000, 3000 and 10007 terms
(coefficients uniform[-1,1]), each compiled under the Horner, Estrin and
Balanced function schemes, each evaluated in FP64 and in compensated FP32 at
2^24 points uniform[-1,1]: 18 evaluations, 1.41e12 term evaluations.

Metric: term evaluations per second (k x points per evaluation), whole job.
Also reported: the roofline of the dominant kernel (the FP64 evaluation,
bound by the FP64 multiply-add issue rate), the plain one-thread-per-point
FP64 Horner kernel on the same FP64 evaluations, an end-to-end figure
through the host-buffer entry point, and the CPU oracle on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (weak scaling, no collective on the data path): launched by
torch.distributed.run, each rank evaluates its own points.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G term-evals/s and roofline fraction vs plain FP64 kernel; p50/p99 serve latency"
UNIT = "G term-evals/s"
KS = (1000, 3000, 10007)
SCHEMES = ("H", "E", "B")
DTYPES = ("f64", "f32c")
NPTS = 1 << 24
SEED = 1000  # configuration index x 1000

# FP64 issue peak: 2 DFMA per clock per SM (GB300) x 152 SMs x 2070 MHz x 2 FLOP
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = 2 * SM_COUNT * SM_MAX_MHZ * 1e6 * 2 / 1e12
FP64_DFMA_GPS = FP64_PEAK_TFLOPS * 1e3 / 2  # 629 G DFMA/s

CPU_SAMPLE_POINTS = 1 << 18  # points per evaluation in the CPU-oracle sample

# Integer-ALU issue roofline of the arithmetic mod p = 2^64 - 2^32 + 1 (the
# mod-p walk and transforms are ALU bound: ncu shows the ALU pipe as the
# busiest).  ALU pipe: 64 lanes per clock per SM (the rate at which ncu's ALU
# utilisation and the measured IMAD chains agree: 64 x 152 x 2070 MHz).
# Minimum ALU-pipe instructions of the method as written: (a b + c) mod p =
# 3 carry additions of the 128-bit product + 2 for the addend + 19 for the
# Goldilocks reduction on 32-bit halves = 24; a radix-2 butterfly = one
# product (22) + a modular addition (9) + a modular subtraction (5) = 36.
# The four 32 x 32 partial products run on the FMA pipe (IMAD), beside them.
ALU_GOPS = 64 * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e9  # 20.1 T ALU lane-ops/s
ALU_OPS_MULADD = 24
ALU_OPS_BUTTERFLY = 36
# Interval walk: 4 directed-rounding FP64 operations per node on the FP64
# pipe (2 lanes per clock per SM, like DFMA)
IV64_NODE_GPS = FP64_DFMA_GPS / 4


def modp_issue_roofline(butterflies, multiplications, rates=None):
    """Time bound of a mod-p workload from the ALU pipe's issue rate."""
    ms = (butterflies * ALU_OPS_BUTTERFLY + multiplications * ALU_OPS_MULADD) / (ALU_GOPS * 1e9) * 1e3
    return {"time_roof_alu_issue": ms,
            "alu_issue_basis": "ALU pipe 64 lanes/clk/SM x 152 x 2070 MHz = %.1f T/s; %d ALU ops per butterfly, "
                               "%d per multiply-add" % (ALU_GOPS / 1e3, ALU_OPS_BUTTERFLY, ALU_OPS_MULADD)}


def workload_config():
    return {
        "workload": "univariate dense, k in {1000, 3000, 10007} terms x schemes {H, E, B} x {f64, f32c}, "
                    "2^24 points uniform[-1,1], coefficients uniform[-1,1]",
        "terms": list(KS),
        "schemes": list(SCHEMES),
        "value_types": list(DTYPES),
        "points": NPTS,
        "term_evals_per_step": sum(KS) * len(SCHEMES) * len(DTYPES) * NPTS,
        "l2": "no flush: each step reads 192 MiB of points and writes 256 MiB of results (> 129 MB L2)",
    }


# ------------------------------------------------------------------ ranks
def points_seed(rank):
    """Each rank evaluates its own points (weak scaling, no data exchange)."""
    return SEED + 1 + 7919 * rank


def combine_ranks(units_per_rank, ms_local, dist=None, device=None):
    """Weak scaling: every rank processed units_per_rank units; the job took as
    long as the slowest rank.  Returns (units of all ranks, max time in ms)."""
    if dist is None:
        return units_per_rank, ms_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return units_per_rank * dist.get_world_size(), float(t.item())


# ------------------------------------------------------------------ CPU oracle
def _oracle_chunk(args):
    k, lo, hi, seed = args
    import workloads as W
    import oracle as O
    e, c, x = W.univariate_case(k, NPTS if hi > NPTS else hi, seed)
    xs = x[:, lo:hi]
    t0 = time.perf_counter()
    O.eval_f64(e, c, xs)                                  # FP64
    O.eval_f64(e, W.to_f32(c).astype(np.float64), W.to_f32(xs).astype(np.float64))  # FP32C reference
    return time.perf_counter() - t0


def cpu_oracle_rate(npoints=CPU_SAMPLE_POINTS):
    """Oracle (plain sum, as it stands) on all host cores: term-evals per second
    over a sample of npoints points of every (k, value type); the plain sum does
    not depend on the scheme, so one sample per k stands for all three schemes."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    chunks = []
    per = max(1, npoints // cores)
    for k in KS:
        for j in range(0, npoints, per):
            chunks.append((k, j, min(npoints, j + per), SEED + k))
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_chunk, [(KS[0], 0, 64, SEED + KS[0])] * cores)  # warm the workers
        t0 = time.perf_counter()
        pool.map(_oracle_chunk, chunks)
        wall = time.perf_counter() - t0
    evals = sum(KS) * npoints * len(DTYPES)  # term-evals actually computed
    return evals / wall, cores, wall


def cpu_oracle_rate_single(npoints=1 << 13):
    """The same oracle in this process, one core: term-evals per second over
    npoints points of every (k, value type)."""
    wall = sum(_oracle_chunk((k, 0, npoints, SEED + k)) for k in KS)
    return sum(KS) * npoints * len(DTYPES) / wall


def run_reference(args):
    """The reference arm: the CPU oracle, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each step: the oracle on 2^16 points of every (k, value type), about half a
    # second of all host cores; the value is the term-evals of all timed steps
    # over their total time
    times = []
    for _ in range(args.warmup):
        cpu_oracle_rate(1 << 12)
    npoints = 1 << 16
    cores = os.cpu_count() or 1
    for _ in range(args.steps):
        _, cores, wall = cpu_oracle_rate(npoints)
        times.append(wall)
    value = sum(KS) * npoints * len(DTYPES) * len(times) / sum(times) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32c", "data": "synthetic",
        "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "2^16 points per (k, value type) per step, schemes share the plain-sum oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while a region runs; the raw CSV goes to
    $FASTPOLY_CLOCKS_CSV when set, else to a temporary file."""

    def __init__(self):
        import tempfile
        self.proc = None
        self.path = os.environ.get("FASTPOLY_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(), "bench_clocks.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, device_index):
        if self.proc is None:
            return None
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9 or f[0] != str(device_index):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    import workloads as W
    import paper_1307_5655_gb300 as fpl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    # inputs resident in HBM; each rank evaluates its own points (weak scaling)
    x64 = W.points_f64(1, NPTS, points_seed(rank))
    d64 = torch.from_numpy(x64).to(dev)
    d32 = torch.from_numpy(W.to_f32(x64)).to(dev)
    out64 = torch.empty(NPTS, dtype=torch.float64, device=dev)
    out32 = torch.empty((2, NPTS), dtype=torch.float32, device=dev)
    trees = []
    for k in KS:
        e, c, _ = W.univariate_case(k, 1, SEED + k)
        for s in SCHEMES:
            trees.append((k, s, fpl.fp_compile(e, c, s)))
    plain_coeffs = {k: torch.from_numpy(W.univariate_case(k, 1, SEED + k)[1][::-1].copy()).to(dev) for k in KS}
    # autotune every (tree, value type) once on a 2^20-point slice (outside the
    # timed region, like compilation); fp_eval then uses the chosen launch
    tuned = {}
    if not args.no_tune:
        for k, s, t in trees:
            tuned["f64/%s/%d" % (s, k)] = fpl.fp_tune(t, "f64", d64[:, : 1 << 20].contiguous())
            tuned["f32c/%s/%d" % (s, k)] = fpl.fp_tune(t, "f32c", d32[:, : 1 << 20].contiguous())

    launches = []  # (kind, k, start_event, end_event)

    def step(record):
        for k, s, t in trees:
            for dt in DTYPES:
                if record:
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                if dt == "f64":
                    fpl.fp_eval(t, "f64", d64, out=out64, stream=stream)
                else:
                    fpl.fp_eval(t, "f32c", d32, out=out32, stream=stream)
                if record:
                    b.record(stream)
                    launches.append((dt, k, a, b, s))

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler()
    if rank == 0:
        clocks.start()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler capture exactly the timed launches
    t_start.record(stream)
    for _ in range(args.steps):
        step(True)
    t_end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = t_start.elapsed_time(t_end)
    clk = clocks.stop(torch.cuda.current_device()) if rank == 0 else None
    units, ms = combine_ranks(workload_config()["term_evals_per_step"] * args.steps, ms, dist, dev)

    # dominant kernel: FP64 evaluation
    f64_ms = sum(a.elapsed_time(b) for dt, k, a, b, _ in launches if dt == "f64")
    f32_ms = sum(a.elapsed_time(b) for dt, k, a, b, _ in launches if dt == "f32c")
    f64_flops = sum(2.0 * k * NPTS for dt, k, a, b, _ in launches if dt == "f64")
    f64_launches = sum(1 for dt, *_ in launches if dt == "f64")
    per_eval = {}
    for dt, k, a, b, s in launches:
        key = "%s/%s/%d" % (dt, s, k)
        per_eval.setdefault(key, []).append(a.elapsed_time(b))
    per_eval = {key: {"ms": float(np.mean(v)), "G_term_evals_per_s": int(key.split("/")[2]) * NPTS / (np.mean(v) * 1e6)}
                for key, v in per_eval.items()}
    achieved = f64_flops / (f64_ms * 1e-3) / 1e12

    # plain FP64 kernel (one thread per point, Horner) on the same FP64 evaluations
    for k in KS:
        fpl.fp_eval_plain_f64(plain_coeffs[k], d64, out=out64, stream=stream)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(len(SCHEMES)):
        for k in KS:
            fpl.fp_eval_plain_f64(plain_coeffs[k], d64, out=out64, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(b)
    plain_rate = len(SCHEMES) * sum(KS) * NPTS / (plain_ms * 1e-3) / 1e9
    ours_f64_rate = f64_flops / 2 / (f64_ms * 1e-3) / 1e9 / args.steps * args.steps

    # end to end through the host-buffer entry point (pinned host memory)
    h64 = torch.from_numpy(x64).pin_memory()
    h32 = torch.from_numpy(W.to_f32(x64)).pin_memory()
    ho64 = torch.empty(NPTS, dtype=torch.float64).pin_memory()
    ho32 = torch.empty((2, NPTS), dtype=torch.float32).pin_memory()

    def e2e_step():
        for k, s, t in trees:
            fpl._check(fpl._lib.fp_eval_host(t.handle, 0, fpl._ptr(h64), NPTS, fpl._ptr(ho64),
                                             fpl._stream_handle(stream)), "fp_eval_host")
            fpl._check(fpl._lib.fp_eval_host(t.handle, 1, fpl._ptr(h32), NPTS, fpl._ptr(ho32),
                                             fpl._stream_handle(stream)), "fp_eval_host")
    e2e_step()
    e2e_steps = max(1, min(args.steps, 2))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = len(trees) * NPTS * (8 + 4)
    d2h = len(trees) * NPTS * (8 + 8)

    value = units / (ms * 1e-3) / 1e9
    e2e_value = workload_config()["term_evals_per_step"] * world / e2e_s / 1e9

    # the other configurations, measured after the timed region (one GPU)
    configs = None
    if world == 1 and not args.no_configs:
        del h64, h32, ho64, ho32
        torch.cuda.empty_cache()
        cfg_clocks = ClockSampler()
        cfg_clocks.start()
        rates = fpl.fp_measure_rates()
        configs = {"config1": measure_config1(fpl, W),
                   "config3": measure_config3(fpl, W, rates, tune=not args.no_tune)}
        torch.cuda.empty_cache()
        configs["config4"] = {
            "workload": "batched composition p o q, 4096 pairs, deg p 512, deg q 64, schemes E and B; MODP exact "
                        "(NTT), FP64 (tensor-core split-precision convolution)",
            "results": measure_compose(fpl, W, 4096, ["modp", "f64"], ["E", "B"], {"modp": 5, "f64": 2}, 1, rates)}
        torch.cuda.empty_cache()
        configs["config5"] = measure_serve(fpl, W, args.serve_requests, args.hbm_budget, overload=False)
        configs["config5"]["workload"] = (
            "serving stream, a stated subsample of %d of the configuration's 100k Poisson requests (same "
            "generator: uni/bivariate, k log-uniform [8, 65536], points log-uniform [1, 2^20], value types "
            "uniform over f64/f32c/iv64/modp)" % args.serve_requests)
        configs["batched_vs_plain_f64"] = measure_batched(fpl, W, 256, args.hbm_budget)
        configs["clocks"] = cfg_clocks.stop(torch.cuda.current_device())

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu:
            rate, cores, wall = cpu_oracle_rate()
            cpu = {"value": rate / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "2^18 points per (k, value type) of the same workload; the plain-sum oracle does not "
                             "depend on the scheme (%.1f s wall)" % wall,
                   "single_thread": {"value": cpu_oracle_rate_single() / 1e9, "unit": UNIT, "cores": 1,
                                     "sample": "2^13 points per (k, value type), in this process"}}
        traffic = f64_traffic_per_launch()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64/f32c", "data": "synthetic", "config": workload_config(),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                         "kernel": "eval_ops_kernel<F64,1,scheme> (FP64 grouped-op walk)",
                         "peak_basis": "derived: 2 DFMA/clk/SM x 152 SMs x 2070 MHz x 2 FLOP (recipe unit counts "
                                       "and max clock); 1 term-eval = 1 multiply + 1 add",
                         "launches": f64_launches, "avg_launch_ms": f64_ms / max(1, f64_launches)},
            "kernel_time_share": {"f64": f64_ms / (f64_ms + f32_ms), "f32c": f32_ms / (f64_ms + f32_ms)},
            "per_evaluation": per_eval,
            "tuned_launch": {key: "%s/ppt%d" % v for key, v in tuned.items()},
            "plain_f64_kernel": {"value": plain_rate, "unit": UNIT,
                                 "ours_f64_same_work": ours_f64_rate,
                                 "speedup": ours_f64_rate / plain_rate},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": len(trees) * len(DTYPES) * args.steps,
            "cpu_baseline": cpu,
            "clocks": clk,
            "configs": configs,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def f64_traffic_per_launch():
    """DRAM bytes (read + written) per launch of the FP64 kernel at 10007
    terms and 2^24 points, from its ncu capture in profiles/, or None."""
    tf = os.path.join(ROOT, "profiles", "eval_f64_traffic.txt")
    if os.path.exists(tf):
        for line in open(tf):
            if line.startswith("bytes_per_launch_k10007_2^24:"):
                return float(line.split(":")[1])
    return None


def run_profile_case(args):
    """One FP64 (or other type) evaluation of a dense polynomial at 2^24 points,
    after one warm-up launch: the small case the ncu captures use."""
    import torch
    import workloads as W
    import paper_1307_5655_gb300 as fpl
    k, scheme, dt = args.profile_k, args.profile_scheme, args.profile_dtype
    torch.cuda.set_device(0)
    # k > 0: dense univariate with k terms at 2^24 points; k = 0: trivariate
    # total degree 40 (12341 terms) at 2^22 points
    nv, npts = (1, NPTS) if k > 0 else (3, 1 << 22)
    if args.profile_points > 0:
        npts = args.profile_points
    x = W.points_f64(nv, npts, SEED + 1)
    if k > 0:
        e, c, _ = W.univariate_case(k, 1, SEED + k)
        em, cm, _ = W.univariate_case(k, 1, SEED + k, "modp")
    else:
        e, c, _ = W.trivariate_case(40, 1, SEED, "f64")
        em, cm, _ = W.trivariate_case(40, 1, SEED, "modp")
    if dt == "modp":
        pts = torch.from_numpy(W.points_modp(nv, npts, SEED + 2).view(np.int64)).cuda()
        t = fpl.fp_compile(em, cm, scheme, modp=True)
    elif dt == "f32c":
        pts = torch.from_numpy(W.to_f32(x)).cuda()
        t = fpl.fp_compile(e, c, scheme)
    elif dt == "iv64":
        lo, hi = W.boxes(nv, npts, SEED + 3)
        pts = torch.from_numpy(np.ascontiguousarray(np.stack([lo, hi], axis=1))).cuda()
        t = fpl.fp_compile(e, c, scheme)
    else:
        pts = torch.from_numpy(x).cuda()
        t = fpl.fp_compile(e, c, scheme)
    for _ in range(2):
        fpl.fp_eval_ex(t, dt, pts, kernel=args.profile_kernel, ppt=args.profile_ppt)
    torch.cuda.synchronize()
    print("profile case done: k=%d scheme=%s dtype=%s kernel=%s ppt=%d points=%d"
          % (k, scheme, dt, args.profile_kernel, args.profile_ppt, npts))


def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def measured_bf16_tflops():
    """Dense bf16 peak of the GB300s (MEASURED_PEAKS.json, burst) or
    the recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def compose_work(t, degq, modp, tc_min=256):
    """Algorithmic operations of one batched composition per pair, following
    the walk's products as the library sizes them.  MODP: (butterflies,
    multiplications) -- a transform of length n is (n/2) log2 n radix-2
    butterflies (one multiplication, one addition, one subtraction each),
    except that the first stage of a zero-padded operand (length <= n/2) is
    n/2 single multiplications; pointwise products, four-step twiddles and
    leaf scalings are single
    multiplications (the inverse transform's 1/n rides on the inverse
    four-step twiddles, or on the cached transform of q^d for n <= 4096,
    scaled once when cached).  FP64: (multiply-adds of the products that run
    on the tensor cores -- both operands at least tc_min long -- , multiply-
    adds of the direct convolutions)."""
    import math
    ex = t.export()
    n_nodes = len(ex["parent"])
    e = ex["node_e"][:, 0].astype(np.int64)
    par, pd = ex["parent"], ex["pd"]
    maxe = e.copy()
    for i in range(n_nodes - 1):
        maxe[par[i]] = max(maxe[par[i]], maxe[i])
    degval = (maxe - e) * degq
    has_child = np.zeros(n_nodes, dtype=bool)
    has_child[par[:-1]] = True
    # powers q^d: closure of the edge degrees under d -> d/2 (even), d-1 (odd)
    need = set(int(d) for d in pd[:-1] if d > 0)
    if pd[-1] > 0:
        need.add(int(pd[-1]))
    stack = list(need)
    while stack:
        d = stack.pop()
        if d > 1:
            m = d // 2 if d % 2 == 0 else d - 1
            if m not in need:
                need.add(m)
                stack.append(m)
    cached = set()
    bfly, mul = 0, 0
    tcmac = 0

    def ntt(n, upper_zero=False):
        # upper_zero: a zero-padded operand (length <= n/2): the first
        # stage's n/2 butterflies are single multiplications (a, a w)
        nonlocal bfly, mul
        bfly += (n // 2) * int(math.log2(n))
        if upper_zero:
            bfly -= n // 2
            mul += n // 2
        if n > 4096:
            mul += n  # four-step twiddles

    def product(alen, blen, bkey):
        nonlocal mul
        nonlocal tcmac
        rl = alen + blen - 1
        if not modp:
            if alen >= tc_min and blen >= tc_min:
                tcmac += alen * blen
            else:
                mul += alen * blen
            return
        n = 1 << max(0, (rl - 1).bit_length())
        ntt(n, 2 * alen <= n)                # forward transform of A
        if (bkey, n) not in cached:          # transform of q^d, once per length
            cached.add((bkey, n))
            ntt(n, 2 * blen <= n)
            if n <= 4096:
                mul += n                     # scaled by 1/n once
        mul += n                             # pointwise
        ntt(n)                               # inverse

    for d in sorted(need):
        if d == 1:
            continue
        if d % 2 == 0:
            product((d // 2) * degq + 1, (d // 2) * degq + 1, d // 2)
        else:
            product((d - 1) * degq + 1, degq + 1, 1)
    for i in range(n_nodes - 1):
        qlen = int(pd[i]) * degq + 1
        if has_child[i]:
            product(int(degval[i]) + 1, qlen, int(pd[i]))
        elif modp:
            mul += qlen                      # leaf: c * q^d
    return (bfly, mul) if modp else (tcmac, mul)


def measure_compose(fpl, W, npairs, dtypes, schemes, steps, warmup, rates):
    """Batched composition: npairs pairs, deg p = 512, deg q = 64 (MODP exact
    by NTT, FP64 by the tensor-core split-precision convolution); per (value
    type, scheme) the time per batch, compositions/s and the roofline."""
    import torch
    degp, degq = 512, 64
    res = {}
    for dt in dtypes:
        pc, qc = W.composition_case(npairs, degp, degq, 4000, dt)
        e = W.dense_univariate_exps(degp + 1)
        if dt == "modp":
            dq = torch.from_numpy(qc.view(np.int64)).cuda()
            dp = torch.from_numpy(np.ascontiguousarray(pc[:, ::-1]).view(np.int64)).cuda()
        else:
            dq = torch.from_numpy(qc).cuda()
            dp = torch.from_numpy(np.ascontiguousarray(pc[:, ::-1])).cuda()
        out = torch.empty((npairs, degp * degq + 1), dtype=torch.int64 if dt == "modp" else torch.float64,
                          device="cuda")
        for s in schemes:
            t = fpl.fp_compile(e, np.ones(degp + 1, dtype=np.uint64 if dt == "modp" else np.float64), s,
                               modp=dt == "modp")
            n_steps = steps[dt] if isinstance(steps, dict) else steps
            ms = _timed(lambda: fpl.fp_compose(t, dt, dq, pcoeffs=dp, out=out), n_steps, warmup)
            bfly, mul = compose_work(t, degq, dt == "modp")
            if dt == "modp":
                roof_ms = npairs * (bfly / rates["modp_butterfly"] + mul / rates["modp_muladd"]) / 1e6
                roof = {"unit": "ms", "butterflies": bfly * npairs, "multiplications": mul * npairs,
                        "butterfly_rate_G_per_s": rates["modp_butterfly"], "mulmod_rate_G_per_s": rates["modp_muladd"],
                        "basis": "measured (fp_measure_rates)"}
                roof.update(modp_issue_roofline(bfly * npairs, mul * npairs, rates))
            else:
                # the tensor-core products: each kept slice pair is one bf16
                # multiply-add per coefficient pair (S (S + 1) / 2 pairs of S =
                # 7 slices); the short products: direct FP64 multiply-adds
                tcmac, dmac = bfly, mul
                pairs = 7 * 8 // 2
                peak, basis = measured_bf16_tflops()
                tc_ms = npairs * tcmac * pairs * 2 / (peak * 1e12) * 1e3
                dfma_ms = npairs * dmac / FP64_DFMA_GPS / 1e6
                roof_ms = tc_ms + dfma_ms
                roof = {"unit": "ms", "bound": "tensor (bf16) + fp64 issue",
                        "tensor_multiply_adds": tcmac * npairs, "slice_pairs": pairs,
                        "bf16_peak_TFLOP_s": peak, "peak_basis": basis, "time_tensor": tc_ms,
                        "direct_multiply_adds": dmac * npairs, "dfma_rate_G_per_s": FP64_DFMA_GPS,
                        "time_direct": dfma_ms,
                        "direct_convolution_time_roof": npairs * (tcmac + dmac) / FP64_DFMA_GPS / 1e6,
                        "basis": "useful slice products (coefficient pairs x kept slice pairs) at the bf16 peak, "
                                 "plus the short products' FP64 multiply-adds at 2 DFMA/clk/SM x 152 x 2070 MHz"}
            roof.update({"time_roof": roof_ms, "time_measured": ms, "frac": roof_ms / ms})
            res["%s/%s" % (dt, s)] = {"ms": ms, "compositions_per_s": npairs / (ms * 1e-3),
                                      "output_coeffs_per_s": npairs * (degp * degq + 1) / (ms * 1e-3),
                                      "roofline": roof}
            t.free()
        del out, dq, dp
        torch.cuda.empty_cache()
    return res


def run_compose(args):
    """Batched composition: 4096 pairs, deg p = 512, deg q = 64 (E and B
    schemes; MODP exact by NTT, FP64 on the tensor cores)."""
    import torch
    import workloads as W
    import paper_1307_5655_gb300 as fpl
    torch.cuda.set_device(0)
    rates = fpl.fp_measure_rates()
    res = measure_compose(fpl, W, args.pairs, args.compose_dtypes.split(","), args.compose_schemes.split(","),
                          args.steps, args.warmup, rates)
    line = {"metric": "compositions/s", "workload": "batched composition, %d pairs, deg p 512, deg q 64" % args.pairs,
            "results": res, "n_gpus": 1, "data": "synthetic"}
    print(json.dumps(line))


def measure_config1(fpl, W):
    """Dense univariate, 1024 terms, Estrin, 65536 points, FP64."""
    import torch
    e, c, x = W.univariate_case(1024, 65536, 1)
    t = fpl.fp_compile(e, c, "E")
    dx = torch.from_numpy(x).cuda()
    out = torch.empty(65536, dtype=torch.float64, device="cuda")
    tune = fpl.fp_tune(t, "f64", dx, out=out)
    ms = _timed(lambda: fpl.fp_eval(t, "f64", dx, out=out), 200, 20)
    # the same evaluation 20 times in a captured CUDA graph: the per-launch
    # cost (a 0.14 ms kernel) is what the graph's replay amortises
    reps = 20
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fpl.fp_eval(t, "f64", dx, out=out)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(reps):
            fpl.fp_eval(t, "f64", dx, out=out)
    ms_graph = _timed(graph.replay, 10, 2) / reps
    rate = 1024 * 65536 / (ms * 1e6)
    rate_graph = 1024 * 65536 / (ms_graph * 1e6)
    t.free()
    return {"workload": "univariate dense, 1024 terms, E, 65536 points uniform[-1,1], FP64", "ms": ms,
            "G_term_evals_per_s": rate, "launch": tune,
            "graph_replay": {"evaluations_per_graph": reps, "ms_per_evaluation": ms_graph,
                             "G_term_evals_per_s": rate_graph, "frac": rate_graph / FP64_DFMA_GPS},
            "roofline": {"bound": "fp64 issue", "peak_G_per_s": FP64_DFMA_GPS, "frac": rate / FP64_DFMA_GPS,
                         "basis": "1 DFMA per term-eval; 2 DFMA/clk/SM x 152 x 2070 MHz"}}


def measure_config3(fpl, W, rates, tune=True):
    """Trivariate total degree 40 (12341 terms) at 2^22 points: intervals
    (width 1e-6 boxes) and residues mod p, under E and B."""
    import torch
    npts = 1 << 22
    res = {}
    e, c, (lo, hi) = W.trivariate_case(40, npts, 300, "iv64")
    dp = torch.from_numpy(np.ascontiguousarray(np.stack([lo, hi], axis=1))).cuda()
    em, cm, xm = W.trivariate_case(40, npts, 301, "modp")
    dm = torch.from_numpy(xm.view(np.int64)).cuda()
    out_iv = torch.empty((2, npts), dtype=torch.float64, device="cuda")
    out_m = torch.empty(npts, dtype=torch.int64, device="cuda")
    for s in ("E", "B"):
        t = fpl.fp_compile(e, c, s)
        lt = fpl.fp_tune(t, "iv64", dp[:, :, : 1 << 18].contiguous()) if tune else None
        ms = _timed(lambda: fpl.fp_eval(t, "iv64", dp, out=out_iv), 3, 1)
        rate = len(e) * npts / (ms * 1e6)
        res["iv64/%s" % s] = {"ms": ms, "G_term_evals_per_s": rate, "launch": lt,
                              "roofline": {"bound": "fp64 issue (directed rounding)", "peak_G_per_s": IV64_NODE_GPS,
                                           "frac": rate / IV64_NODE_GPS,
                                           "frac_of_measured_rd_rate": rate / (rates["dadd_rd"] / 4),
                                           "basis": "4 directed-rounding FP64 ops per node at 2 per clk per SM"}}
        t.free()
        tm = fpl.fp_compile(em, cm, s, modp=True)
        lt = fpl.fp_tune(tm, "modp", dm[:, : 1 << 20].contiguous()) if tune else None
        ms = _timed(lambda: fpl.fp_eval(tm, "modp", dm, out=out_m), 5, 1)
        rate = len(em) * npts / (ms * 1e6)
        peak = ALU_GOPS / ALU_OPS_MULADD
        res["modp/%s" % s] = {"ms": ms, "G_term_evals_per_s": rate, "launch": lt,
                              "roofline": {"bound": "integer ALU issue", "peak_G_per_s": peak, "frac": rate / peak,
                                           "frac_of_measured_muladd_rate": rate / rates["modp_muladd"],
                                           "basis": "%d ALU-pipe ops per (a b + c) mod p at 64 lanes/clk/SM"
                                                    % ALU_OPS_MULADD}}
        tm.free()
    return res


def serve_requests(fpl, W, n, seed=5000):
    """The serving stream's requests: uni/bivariate polynomials with term count
    log-uniform in [8, 65536] (bivariate: the first k monomials in graded
    order), point count log-uniform in [1, 2^20], value type uniform over FP64 /
    FP32C / IV64 / MODP; scheme E (B when k is not a power of two).  Trees are
    compiled once and stay resident (8 per value type and variable count);
    points and results live in pinned host pools.  Returns (requests, term-evals,
    trees)."""
    import torch
    r = W.rng(seed)
    dts = ["f64", "f32c", "iv64", "modp"]
    maxp = 1 << 20
    pools, trees = {}, {}
    for dt in dts:
        for nv in (1, 2):
            cnt = maxp * nv * (2 if dt == "iv64" else 1)
            npdt = {"f64": np.float64, "f32c": np.float32, "iv64": np.float64, "modp": np.uint64}[dt]
            buf = torch.empty(cnt, dtype=torch.float64 if npdt in (np.float64,) else
                              (torch.float32 if npdt == np.float32 else torch.int64), pin_memory=True).numpy()
            if dt == "modp":
                buf = buf.view(np.uint64)
                buf[:] = W.residues(cnt, 11 + nv)
            else:
                buf[:] = W.uniform_f64(cnt, 13 + nv).astype(npdt)
            pools[(dt, nv)] = buf
            lst = []
            for i in range(8):
                k = int(np.exp(r.uniform(np.log(8), np.log(65536))))
                e = W.dense_univariate_exps(k) if nv == 1 else W.graded_prefix_exps(k, 2)
                c = W.residues(len(e), 100 + i) if dt == "modp" else W.uniform_f64(len(e), 100 + i)
                lst.append((fpl.fp_compile(e, c, "E" if (k & (k - 1)) == 0 else "B", modp=dt == "modp"), len(e)))
            trees[(dt, nv)] = lst
    outs = {}
    for dt in dts:
        npdt = {"f64": np.float64, "f32c": np.float32, "iv64": np.float64, "modp": np.uint64}[dt]
        t = torch.empty(2 * maxp * (2 if npdt == np.float32 else 1), dtype=torch.float64, pin_memory=True).numpy()
        outs[dt] = t.view(npdt)
    reqs = []
    for j in range(n):
        dt = dts[int(r.integers(0, 4))]
        nv = 1 + int(r.integers(0, 2))
        tree, k = trees[(dt, nv)][int(r.integers(0, 8))]
        npts = int(np.exp(r.uniform(0, np.log(maxp))))
        per = nv * (2 if dt == "iv64" else 1)
        pts = pools[(dt, nv)][: per * npts].reshape((nv, 2, npts) if dt == "iv64" else (nv, npts))
        shp = fpl.out_shape(dt, npts)
        out = outs[dt][: int(np.prod(shp))].reshape(shp)
        reqs.append((tree, dt, pts, out, k * npts))
    return reqs, sum(x[4] for x in reqs), trees


def measure_serve(fpl, W, n, hbm_budget_mib=8192, seed=5000, overload=True, isolated=True):
    """Continuous batching on the request stream: saturated throughput (all
    submitted at once), Poisson arrivals at 0.7 x that rate (p50/p99 latency,
    slowdown against each request's own isolated time), an overload stream at
    1.2 x, and one launch per request (fp_eval_host in turn)."""
    reqs, total_evals, _trees = serve_requests(fpl, W, n, seed)

    def serve(arrivals):
        srv = fpl.Server(hbm_budget_bytes=hbm_budget_mib << 20, max_batch_jobs=256, streams=4)
        done, tickets = {}, []
        t0 = time.perf_counter()
        for (tree, dt, pts, out, _), ta in zip(reqs, arrivals):
            if ta is not None:
                while time.perf_counter() - t0 < ta:
                    pass
            tickets.append(srv.submit(tree, dt, pts, out))
            done.update({x[0]: x[2] for x in srv.poll()})
        srv.drain(3600)
        wall = time.perf_counter() - t0
        done.update({x[0]: x[2] for x in srv.poll()})
        st = srv.stats()
        srv.close()
        return wall, np.array([done.get(tk, np.nan) for tk in tickets], dtype=np.float64), st

    serve([None] * min(8, len(reqs)))  # warm the server path
    wall_sat, _lat_sat, st_sat = serve([None] * len(reqs))
    rate = len(reqs) / wall_sat
    gaps = W.rng(seed + 1).exponential(1.0 / (0.7 * rate), size=len(reqs))
    wall_open, lat_open, st_open = serve(list(np.cumsum(gaps)))
    lat_open = np.where(np.isnan(lat_open), np.nanmax(lat_open), lat_open)
    res = {
        "requests": len(reqs), "term_evals": int(total_evals),
        "saturated": {"wall_s": wall_sat, "requests_per_s": rate, "G_term_evals_per_s": total_evals / wall_sat / 1e9,
                      "batches": st_sat["batches"], "peak_hbm_bytes": st_sat["peak_bytes"]},
        "poisson_0.7": {"rate_per_s": 0.7 * rate, "wall_s": wall_open,
                        "p50_ms": float(np.percentile(lat_open, 50)) / 1e3,
                        "p99_ms": float(np.percentile(lat_open, 99)) / 1e3,
                        "G_term_evals_per_s": total_evals / wall_open / 1e9, "batches": st_open["batches"]},
        "hbm_budget_MiB": hbm_budget_mib,
    }
    if overload:
        wall_over, lat_over, st_over = serve(list(np.cumsum(gaps * (0.7 / 1.2))))
        lat_over = np.where(np.isnan(lat_over), np.nanmax(lat_over), lat_over)
        res["overload_1.2"] = {"rate_per_s": 1.2 * rate, "wall_s": wall_over,
                               "p50_ms": float(np.percentile(lat_over, 50)) / 1e3,
                               "p99_ms": float(np.percentile(lat_over, 99)) / 1e3,
                               "G_term_evals_per_s": total_evals / wall_over / 1e9, "batches": st_over["batches"],
                               "peak_hbm_bytes": st_over["peak_bytes"]}
    if isolated:
        iso = np.empty(len(reqs))
        t0 = time.perf_counter()
        for i, (tree, dt, pts, out, _) in enumerate(reqs):
            ti = time.perf_counter()
            fpl.fp_eval_host(tree, dt, pts)
            iso[i] = (time.perf_counter() - ti) * 1e6
        wall_seq = time.perf_counter() - t0
        slow = lat_open / iso
        res["poisson_0.7"].update({"slowdown_p50": float(np.nanpercentile(slow, 50)),
                                   "slowdown_p99": float(np.nanpercentile(slow, 99)),
                                   "slowdown_note": "latency / the request's own run time alone (fp_eval_host)"})
        res["one_launch_per_request"] = {"wall_s": wall_seq, "requests_per_s": len(reqs) / wall_seq,
                                         "G_term_evals_per_s": total_evals / wall_seq / 1e9,
                                         "continuous_batching_speedup": wall_seq / wall_sat}
    return res


def run_compose_accuracy(args):
    """FP64 composition, 4096 pairs of deg p 512 and deg q 64 (schemes E and
    B): time and error against the oracle (8 sampled pairs) for the tensor-core
    products with 6, 7 and 8 slices and for the direct FP64 convolution.
    Errors are |r - oracle| over s = |p| o |q|, the plain walk on absolute
    values: componentwise (max over coefficients of err_i / s_i), local (over
    the maximum of s within +-128 coefficients: the tensor path's blockwise
    bar) and normwise (max err over max s)."""
    import os as _os
    from concurrent.futures import ThreadPoolExecutor
    import torch
    import workloads as W
    import oracle as O
    import paper_1307_5655_gb300 as fpl
    from scipy.ndimage import maximum_filter1d
    torch.cuda.set_device(0)
    npairs, degp, degq = args.pairs, 512, 64
    pc, qc = W.composition_case(npairs, degp, degq, 4000, "f64")
    js = np.sort(W.rng(17).choice(npairs, 8, replace=False))
    with ThreadPoolExecutor(max_workers=_os.cpu_count() or 1) as ex:
        ref = list(ex.map(lambda j: O.compose_f64(pc[j], qc[j]), js))
    dq = torch.from_numpy(qc).cuda()
    dp = torch.from_numpy(np.ascontiguousarray(pc[:, ::-1])).cuda()
    out = torch.empty((npairs, degp * degq + 1), dtype=torch.float64, device="cuda")
    e = W.dense_univariate_exps(degp + 1)
    res = {}
    for s in args.compose_schemes.split(","):
        t = fpl.fp_compile(e, np.ones(degp + 1), s)
        for name, (slices, min_len) in (("tc6", (6, 0)), ("tc7", (7, 0)), ("tc8", (8, 0)), ("direct", (0, -1))):
            fpl.fp_set_compose_f64(slices, min_len)
            ms = _timed(lambda: fpl.fp_compose(t, "f64", dq, pcoeffs=dp, out=out), 1 if name == "direct" else 2, 1)
            got = out[torch.from_numpy(js).cuda()].cpu().numpy()
            comp, loc, norm = 0.0, 0.0, 0.0
            for row, (want, absw) in zip(got, ref):
                err = np.abs(row - want)
                nz = absw > 1e-290
                comp = max(comp, float((err[nz] / absw[nz]).max()))
                locs = maximum_filter1d(absw, size=257, mode="constant", cval=0.0)
                loc = max(loc, float((err / np.maximum(locs, 1e-300)).max()))
                norm = max(norm, float(err.max() / absw.max()))
            res["%s/%s" % (s, name)] = {"ms": ms, "compositions_per_s": npairs / (ms * 1e-3),
                                        "err_componentwise_max": comp, "err_local_max": loc,
                                        "err_normwise_max": norm}
        t.free()
    fpl.fp_set_compose_f64(0, 0)
    print(json.dumps({"metric": "FP64 composition time and error vs oracle per product method",
                      "workload": "%d pairs, deg p 512, deg q 64 (q uniform[-1,1]/65), 8 sampled pairs" % npairs,
                      "error_basis": "err / s, s = |p| o |q| (componentwise over s_i > 1e-290; local over max s "
                                     "within +-128; normwise over max s)", "u": 2.0 ** -53, "results": res}))


def run_eval_config(args):
    """Per-configuration evaluation measurements: dense univariate 1024 terms at
    65536 points (E), trivariate total degree 40 at 2^22 points (IV64, MODP,
    and FP64 / FP32C for the grouped-op kernel on a multivariate tree)."""
    import torch
    import workloads as W
    import paper_1307_5655_gb300 as fpl
    torch.cuda.set_device(0)
    res = {}
    e, c, x = W.univariate_case(1024, 65536, 1)
    t = fpl.fp_compile(e, c, "E")
    dx = torch.from_numpy(x).cuda()
    ms = _timed(lambda: fpl.fp_eval(t, "f64", dx), 50, 5)
    res["univariate_1024_E_f64_65536pts"] = {"ms": ms, "G_term_evals_per_s": 1024 * 65536 / (ms * 1e6)}
    npts = 1 << 22
    for s in ("E", "B"):
        e, c, (lo, hi) = W.trivariate_case(40, npts, 300, "iv64")
        t = fpl.fp_compile(e, c, s)
        dp = torch.from_numpy(np.ascontiguousarray(np.stack([lo, hi], axis=1))).cuda()
        tune = fpl.fp_tune(t, "iv64", dp[:, :, : 1 << 18].contiguous()) if not args.no_tune else None
        ms = _timed(lambda: fpl.fp_eval(t, "iv64", dp), 2, 1)
        res["trivariate_deg40_%s_iv64_2^22" % s] = {"ms": ms, "G_term_evals_per_s": len(e) * npts / (ms * 1e6),
                                                     "launch": tune}
        em, cm, xm = W.trivariate_case(40, npts, 301, "modp")
        tm = fpl.fp_compile(em, cm, s, modp=True)
        dm = torch.from_numpy(xm.view(np.int64)).cuda()
        tune = fpl.fp_tune(tm, "modp", dm[:, : 1 << 20].contiguous()) if not args.no_tune else None
        ms = _timed(lambda: fpl.fp_eval(tm, "modp", dm), 3, 1)
        res["trivariate_deg40_%s_modp_2^22" % s] = {"ms": ms, "G_term_evals_per_s": len(em) * npts / (ms * 1e6),
                                                     "launch": tune}
        ef, cf, xf = W.trivariate_case(40, npts, 302, "f64")
        tf = fpl.fp_compile(ef, cf, s)
        df = torch.from_numpy(xf).cuda()
        for dt, d in (("f64", df), ("f32c", torch.from_numpy(W.to_f32(xf)).cuda())):
            tune = fpl.fp_tune(tf, dt, d[:, : 1 << 20].contiguous()) if not args.no_tune else None
            ms = _timed(lambda: fpl.fp_eval(tf, dt, d), 3, 1)
            res["trivariate_deg40_%s_%s_2^22" % (s, dt)] = {"ms": ms, "G_term_evals_per_s": len(ef) * npts / (ms * 1e6),
                                                           "launch": tune}
    # sparse trivariate: a seeded 30 % of the degree-40 monomials, so groups
    # miss their lowest terms and the tree carries zero-coefficient virtual
    # roots (the multivariate reading of the Remark of Sec. 1.1)
    full = W.total_degree_exps(3, 40)
    keep = W.rng(303).random(len(full)) < 0.3
    es = full[keep]
    for s in ("E", "B"):
        cs = W.uniform_f64(len(es), 304)
        xs = W.points_f64(3, npts, 305)
        ts = fpl.fp_compile(es, cs, s)
        info = ts.info()
        ds = torch.from_numpy(xs).cuda()
        tune = fpl.fp_tune(ts, "f64", ds[:, : 1 << 20].contiguous()) if not args.no_tune else None
        ms = _timed(lambda: fpl.fp_eval(ts, "f64", ds), 3, 1)
        res["sparse_trivariate_30pct_%s_f64_2^22" % s] = {
            "ms": ms, "terms": int(len(es)), "nodes": info["nnodes"],
            "virtual_nodes": int(info["nnodes"] - len(es)),
            "G_term_evals_per_s": len(es) * npts / (ms * 1e6),
            "G_node_evals_per_s": info["nnodes"] * npts / (ms * 1e6), "launch": tune}
    print(json.dumps({"metric": "G term-evals/s", "results": res, "n_gpus": 1, "data": "synthetic"}))


def run_serve(args):
    """Serving stream (serve_requests): saturated throughput, Poisson arrivals
    at 0.7 x that rate with p50/p99 latency, an overload stream at 1.2 x, and
    the same requests served one launch at a time (fp_eval_host per request)."""
    import torch
    import workloads as W
    import paper_1307_5655_gb300 as fpl
    torch.cuda.set_device(0)
    res = measure_serve(fpl, W, args.requests, args.hbm_budget)
    line = {"metric": "p50/p99 serve latency and throughput",
            "workload": "%d requests, uni/bivariate, k log-uniform [8, 65536], points log-uniform [1, 2^20], "
                        "value types uniform over f64/f32c/iv64/modp" % args.requests,
            "n_gpus": 1, "data": "synthetic"}
    line.update(res)
    print(json.dumps(line))


def run_accuracy(args):
    """Error of the FP64 and compensated FP32 paths against the oracle per
    (k, scheme) of the benchmark workload, on a sample of 4096 of its points:
    max and median of |r - p| / sum |c_e x^e| (the condition scale)."""
    import torch
    import workloads as W
    import oracle as O
    import paper_1307_5655_gb300 as fpl
    torch.cuda.set_device(0)
    x = W.points_f64(1, NPTS, points_seed(0))
    idx = np.sort(W.rng(9).choice(NPTS, 4096, replace=False))
    d64 = torch.from_numpy(x).cuda()
    d32 = torch.from_numpy(W.to_f32(x)).cuda()
    res = {}
    for k in KS:
        e, c, _ = W.univariate_case(k, 1, SEED + k)
        want, S = O.eval_f64(e, c, x[:, idx])
        c32 = W.to_f32(c).astype(np.float64)
        want32, S32 = O.eval_f64(e, c32, W.to_f32(x[:, idx]).astype(np.float64))
        for s in SCHEMES:
            t = fpl.fp_compile(e, c, s)
            g = fpl.fp_eval(t, "f64", d64).cpu().numpy()[idx]
            g32 = fpl.fp_eval(t, "f32c", d32).cpu().numpy()[:, idx]
            r64 = np.abs(g - want) / S
            r32 = np.abs(g32[0].astype(np.float64) + g32[1].astype(np.float64) - want32) / S32
            plain32 = np.abs(g32[0].astype(np.float64) - want32) / S32
            res["%s/%d" % (s, k)] = {
                "f64_max": float(r64.max()), "f64_median": float(np.median(r64)),
                "f64_bound_4nu": 4 * (k - 1) * 2.0 ** -53,
                "f32c_max": float(r32.max()), "f32c_median": float(np.median(r32)),
                "f32c_hi_only_median": float(np.median(plain32)),
            }
    print(json.dumps({"metric": "relative error vs oracle (scaled by sum |c_e x^e|)", "sample_points": 4096,
                      "results": res}))


def run_staircase(args):
    """The paper's staircase (Sec. 1.2, Sec. 3): composition time around a
    power-of-two term count, Estrin vs Balanced, mod p, deg q = 64."""
    import torch
    import workloads as W
    import paper_1307_5655_gb300 as fpl
    torch.cuda.set_device(0)
    npairs, degq = args.pairs, 64
    res = {}
    for terms in (254, 255, 256, 257, 258, 510, 511, 512, 513, 514):
        degp = terms - 1
        pc, qc = W.composition_case(npairs, degp, degq, 7000 + terms, "modp")
        dq = torch.from_numpy(qc.view(np.int64)).cuda()
        dp = torch.from_numpy(np.ascontiguousarray(pc[:, ::-1]).view(np.int64)).cuda()
        out = torch.empty((npairs, degp * degq + 1), dtype=torch.int64, device="cuda")
        e = W.dense_univariate_exps(terms)
        for s in ("E", "B"):
            t = fpl.fp_compile(e, np.ones(terms, dtype=np.uint64), s, modp=True)
            ms = _timed(lambda: fpl.fp_compose(t, "modp", dq, pcoeffs=dp, out=out), args.steps, 1)
            res["%s/%d" % (s, terms)] = ms
    print(json.dumps({"metric": "ms per batch of %d compositions mod p, deg q %d" % (npairs, degq),
                      "results": res}))


def measure_batched(fpl, W, n, hbm_budget_mib=8192):
    """Many FP64 univariate polynomials of uneven size -- the FP64 univariate
    part of the serving mix: k log-uniform in [8, 65536] dense terms, points
    log-uniform in [1, 2^20], coefficients and points uniform[-1, 1], scheme E
    (B when k is not a power of two) -- the batched and served forms against
    the plain one-launch-per-polynomial FP64 kernel (one thread per point,
    Horner) on the same inputs.  Device-resident: one fp_eval_batch call (it
    plans the batch every call), a planned batch (fp_batch_create once,
    launch only), and the plain kernel once per polynomial back to back on
    one stream.  Host buffers (pinned): the server (submit all, drain) and the
    plain kernel once per polynomial with its copy in and copy out on one
    stream.  Wall time around each pass (synchronized), median of 3 after a
    warm-up pass; every result is checked against the plain kernel's within
    8 k u S (S = sum |c_e| |x|^e, both are FP64 evaluations within 4 k u S)."""
    import torch
    r = W.rng(6000)
    polys = []
    for i in range(n):
        k = int(np.exp(r.uniform(np.log(8), np.log(65536))))
        npts = int(np.exp(r.uniform(0, np.log(1 << 20))))
        e, c, x = W.univariate_case(k, npts, 6100 + i)
        t = fpl.fp_compile(e, c, "E" if (k & (k - 1)) == 0 else "B")
        polys.append((k, npts, t, c, x))
    evals = sum(k * m for k, m, _, _, _ in polys)
    dev = torch.device("cuda")
    coef_d = [torch.from_numpy(c[::-1].copy()).to(dev) for _, _, _, c, _ in polys]
    pts_d = [torch.from_numpy(x).to(dev) for _, _, _, _, x in polys]
    out_plain = [torch.empty(m, dtype=torch.float64, device=dev) for _, m, _, _, _ in polys]
    out_batch = [torch.empty((1, m), dtype=torch.float64, device=dev) for _, m, _, _, _ in polys]
    jobs = [(t, pts_d[i], out_batch[i]) for i, (_, _, t, _, _) in enumerate(polys)]
    pts_h = [torch.from_numpy(x).pin_memory() for _, _, _, _, x in polys]
    out_h = [torch.empty(m, dtype=torch.float64).pin_memory() for _, m, _, _, _ in polys]
    out_srv = [torch.empty((1, m), dtype=torch.float64).pin_memory().numpy() for _, m, _, _, _ in polys]

    def wall(fn):
        ts = []
        for rep in range(4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            if rep:
                ts.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(ts))

    def plain_device():
        for i in range(n):
            fpl.fp_eval_plain_f64(coef_d[i], pts_d[i], out=out_plain[i])

    def batch_call():
        fpl.fp_eval_batch("f64", jobs)

    planned = fpl.Batch("f64", jobs)

    def plain_host():
        for i in range(n):
            d = pts_h[i].to(dev, non_blocking=True)
            o = fpl.fp_eval_plain_f64(coef_d[i], d)
            out_h[i].copy_(o, non_blocking=True)

    srv = fpl.Server(hbm_budget_bytes=hbm_budget_mib << 20, max_batch_jobs=256, streams=4)
    pts_srv = [p.numpy() for p in pts_h]

    def served():
        for i, (_, _, t, _, _) in enumerate(polys):
            srv.submit(t, "f64", pts_srv[i], out_srv[i])
        srv.drain(3600)
        done = srv.poll()
        assert len(done) == n and all(st == 0 for _, st, _ in done), "server requests failed"

    # the resident kernel: every polynomial submitted into the running kernel
    # (device-resident inputs), waiting for all
    out_res = [torch.empty((1, m), dtype=torch.float64, device=dev) for _, m, _, _, _ in polys]
    items = sum(-(-(-(-m // 128)) // 4) for _, m, _, _, _ in polys)  # work items of one pass (4 tiles of 128 points)
    resident = fpl.Resident("f64", max_jobs=5 * n + 64, idle_exit_s=1.0, max_items=5 * items + 64)
    torch.cuda.synchronize()

    def resident_pass():
        tk = [resident.submit(t, pts_d[i], out_res[i]) for i, (_, _, t, _, _) in enumerate(polys)]
        for x in tk:
            resident.wait(x, 600.0)

    def wall_resident():
        # the resident kernel stays on its own stream until its idle timeout:
        # a device-wide synchronize would wait for that; the pass is timed
        # from the first submission to the last completion
        ts = []
        for rep in range(4):
            torch.cuda.current_stream().synchronize()
            t0 = time.perf_counter()
            resident_pass()
            if rep:
                ts.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(ts))

    res = {"resident_kernel_ms": wall_resident()}
    res.update({"plain_one_launch_per_poly_ms": wall(plain_device), "fp_eval_batch_ms": wall(batch_call),
                "planned_batch_launch_ms": wall(planned.launch)})
    res["speedup_fp_eval_batch"] = res["plain_one_launch_per_poly_ms"] / res["fp_eval_batch_ms"]
    res["speedup_planned_batch"] = res["plain_one_launch_per_poly_ms"] / res["planned_batch_launch_ms"]
    res["speedup_resident_kernel"] = res["plain_one_launch_per_poly_ms"] / res["resident_kernel_ms"]
    # admission latency of a small job (100 terms, 1000 points): submitted to
    # the running resident kernel, against a launch of fp_eval with a synchronize
    e_s, c_s, x_s = W.univariate_case(100, 1000, 6050)
    t_s = fpl.fp_compile(e_s, c_s, "B")
    d_s = torch.from_numpy(x_s).to(dev)
    o_s = torch.empty((1, 1000), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    lat_res, lat_launch = [], []
    for _ in range(50):
        t0 = time.perf_counter()
        resident.wait(resident.submit(t_s, d_s, o_s), 60.0)
        lat_res.append((time.perf_counter() - t0) * 1e6)
    resident.close()  # stops the kernel (the synchronizes below would wait for its idle timeout)
    for _ in range(50):
        t0 = time.perf_counter()
        fpl.fp_eval(t_s, "f64", d_s, out=o_s[0])
        torch.cuda.synchronize()
        lat_launch.append((time.perf_counter() - t0) * 1e6)
    res["small_job_latency_us"] = {"resident_kernel_median": float(np.median(lat_res)),
                                   "launch_and_sync_median": float(np.median(lat_launch)),
                                   "job": "100 terms, 1000 points, FP64"}
    host = {"plain_with_copies_ms": wall(plain_host), "server_ms": wall(served)}
    host["speedup_server"] = host["plain_with_copies_ms"] / host["server_ms"]
    # the results agree within the FP64 bound
    worst = 0.0
    for i, (k, m, _, c, x) in enumerate(polys):
        S = fpl.fp_eval_plain_f64(coef_d[i].abs(), pts_d[i].abs()).cpu().numpy()
        ref = out_plain[i].cpu().numpy()
        for got in (out_batch[i][0].cpu().numpy(), out_h[i].numpy(), out_srv[i][0], out_res[i][0].cpu().numpy()):
            worst = max(worst, float(np.max(np.abs(got - ref) / (8 * k * 2.0 ** -53 * S + 1e-300))))
    planned.free()
    srv.close()
    line = {"metric": "ms per batch of %d FP64 polynomials of uneven size" % n,
            "workload": "univariate dense, k log-uniform [8, 65536], points log-uniform [1, 2^20], "
                        "E (B for k not a power of two), uniform[-1, 1]",
            "term_evals": int(evals), "device_resident": res, "host_buffers": host,
            "G_term_evals_per_s": {"plain": evals / res["plain_one_launch_per_poly_ms"] / 1e6,
                                   "fp_eval_batch": evals / res["fp_eval_batch_ms"] / 1e6,
                                   "planned_batch": evals / res["planned_batch_launch_ms"] / 1e6,
                                   "resident_kernel": evals / res["resident_kernel_ms"] / 1e6,
                                   "server_host_buffers": evals / host["server_ms"] / 1e6,
                                   "plain_host_buffers": evals / host["plain_with_copies_ms"] / 1e6},
            "max_error_over_8kuS": worst, "n_gpus": 1, "data": "synthetic"}
    return line


def run_batched(args):
    """measure_batched on --batch-polys polynomials (one JSON line)."""
    import torch
    import workloads as W
    import paper_1307_5655_gb300 as fpl
    torch.cuda.set_device(0)
    print(json.dumps(measure_batched(fpl, W, args.batch_polys, args.hbm_budget)))


def run_peaks(args):
    """Roofline denominators measured with the library's own arithmetic
    (fp_measure_rates), with the SM clock sampled while they run."""
    import torch
    import paper_1307_5655_gb300 as fpl
    torch.cuda.set_device(0)
    fpl.fp_measure_rates()  # warm-up (clocks ramp)
    mon = ClockSampler()
    mon.start()
    rates = fpl.fp_measure_rates()
    clocks = mon.stop(torch.cuda.current_device())
    derived = {
        "fp64_node_roofline_G_per_s": rates["dfma"],
        "f32c_node_roofline_G_per_s (general form)": rates["f32c_mad"],
        "f32c_horner_node_roofline_G_per_s": rates["f32c_horner"],
        "modp_node_roofline_G_per_s": rates["modp_muladd"],
        "iv64_node_roofline_G_per_s (4 directed-rounding FP64 operations)": rates["dadd_rd"] / 4,
    }
    print(json.dumps({"metric": "sustained G op/s per operation (roofline denominators)", "rates": rates,
                      "per_node": derived, "clocks": clocks, "n_gpus": 1}))


def run_rns(args):
    """Exact integer evaluation through residues (the paper's multi-precision
    setting, Sec. 3): dense univariate integer polynomials with random signed
    coefficients of cbits bits at 2^16 random signed points of xbits bits;
    as many primes q = 2^64 - c as the values need; the walk modulo every
    prime in one launch, then the Chinese remainder reconstruction.  The CPU
    baseline is the oracle's exact integer sum (Python integers) on a sample."""
    import time
    import torch
    import workloads as W
    import paper_1307_5655_gb300 as fpl
    from oracle import exact as X
    torch.cuda.set_device(0)
    npts = 1 << 16
    res = {}
    for deg, cbits, xbits in ((100, 256, 32), (60, 1024, 32), (30, 128, 100), (1000, 64, 3)):
        k = deg + 1
        r = W.rng(7000 + deg)
        coeffs = [int(v) * (1 if r.random() < 0.5 else -1) for v in
                  (int.from_bytes(r.bytes((cbits + 7) // 8), "little") >> (8 * ((cbits + 7) // 8) - cbits)
                   for _ in range(k))]
        xs = [int(v) - (1 << (xbits - 1)) for v in
              (int.from_bytes(r.bytes((xbits + 7) // 8), "little") >> (8 * ((xbits + 7) // 8) - xbits)
               for _ in range(npts))]
        nq = (cbits + deg * xbits + k.bit_length() + 2 + 63) // 64 + 1
        qs = [int(v) for v in fpl.fp_rns_primes(nq)]
        e = W.dense_univariate_exps(k)
        resid = np.array([[c % q for c in coeffs] for q in qs], dtype=np.uint64)
        pts = np.array([[[x % q for x in xs]] for q in qs], dtype=np.uint64)
        t = fpl.fp_compile_rns(e, resid, "E")
        d = torch.from_numpy(pts.view(np.int64)).cuda()
        out = torch.empty((nq, npts), dtype=torch.int64, device="cuda")
        limbs = torch.empty((npts, nq), dtype=torch.int64, device="cuda")
        ms_eval = _timed(lambda: fpl.fp_eval_rns(t, d, out=out), args.steps, args.warmup)
        ms_crt = _timed(lambda: fpl.fp_crt(out, out=limbs), args.steps, args.warmup)
        # spot check against the oracle
        lim = limbs.cpu().numpy().view(np.uint64)
        for j in (0, npts // 2, npts - 1):
            assert fpl.limbs_to_int(lim[j]) == X.int_value(e.tolist(), coeffs, (xs[j],))
        nsample = 64 if deg * xbits <= 4000 else 16
        t0 = time.perf_counter()
        for j in range(nsample):
            X.int_value(e.tolist(), coeffs, (xs[j],))
        cpu_s = (time.perf_counter() - t0) / nsample
        total_ms = ms_eval + ms_crt
        res["deg%d_c%db_x%db" % (deg, cbits, xbits)] = {
            "primes": nq, "value_bits": nq * 64, "eval_ms": ms_eval, "crt_ms": ms_crt,
            "bigint_evals_per_s": npts / (total_ms * 1e-3),
            "G_modular_term_evals_per_s": nq * k * npts / (ms_eval * 1e6),
            "cpu_oracle_bigint_evals_per_s_1core": 1.0 / cpu_s, "cpu_sample_points": nsample}
        t.free()
    print(json.dumps({"metric": "exact big-integer evaluations/s", "points": npts, "scheme": "E",
                      "results": res, "n_gpus": 1, "data": "synthetic"}))


def run_hybrid(args):
    """The paper's combined scheme (Remark of Sec. 1.1): Estrin above k0 terms,
    Horner below, against H, E and B, FP64 and compensated FP32, k = 10007 at
    2^24 points (each tree autotuned)."""
    import math
    import torch
    import workloads as W
    import paper_1307_5655_gb300 as fpl
    torch.cuda.set_device(0)
    k = 10007
    x = W.points_f64(1, NPTS, points_seed(0))
    d64 = torch.from_numpy(x).cuda()
    d32 = torch.from_numpy(W.to_f32(x)).cuda()
    e, c, _ = W.univariate_case(k, 1, SEED + k)
    res = {}
    variants = [("H", None), ("E", None), ("B", None), ("D", None)]
    for k0 in (4, 8, 16, 32, 64, 128, 512):
        ft = np.ones(k + 1, dtype=np.int32)
        for n in range(1, k + 1):
            ft[n] = 2 ** int(math.floor(math.log2(n))) if n + 1 > k0 else 1
        variants.append(("hybrid_k0_%d" % k0, ft))
    for name, ft in variants:
        t = fpl.fp_compile(e, c, "CUSTOM" if ft is not None else name, ft)
        for dt, d in (("f64", d64), ("f32c", d32)):
            fpl.fp_tune(t, dt, d[:, : 1 << 20].contiguous())
            ms = _timed(lambda: fpl.fp_eval(t, dt, d), 3, 1)
            res["%s/%s" % (dt, name)] = {"ms": ms, "G_term_evals_per_s": k * NPTS / (ms * 1e6)}
    # the scheme autotuner (fp_tune_scheme) on a 2^20-point sample, then the
    # chosen tree timed at full size
    chosen = {}
    for dt, d in (("f64", d64), ("f32c", d32)):
        t, k0 = fpl.fp_tune_scheme(e, c, dt, d[:, : 1 << 20].contiguous())
        ms = _timed(lambda: fpl.fp_eval(t, dt, d), 3, 1)
        chosen[dt] = {"k0": k0, "meaning": "Balanced" if k0 == 0 else ("Horner" if k0 >= k else "Estrin above k0 terms"),
                      "ms": ms, "G_term_evals_per_s": k * NPTS / (ms * 1e6)}
        t.free()
    print(json.dumps({"metric": "G term-evals/s", "workload": "k = 10007, 2^24 points", "results": res,
                      "fp_tune_scheme": chosen}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="univariate", choices=["univariate", "compose", "compose-accuracy",
                                                                "eval-configs", "serve", "accuracy",
                                                                "staircase", "hybrid", "peaks", "rns", "batched"],
                    help="univariate: the benchmark line; the others print their own measurement line")
    ap.add_argument("--pairs", type=int, default=4096)
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--batch-polys", type=int, default=256, help="polynomials of --workload batched")
    ap.add_argument("--hbm-budget", type=int, default=8192, help="MiB of device memory for requests in flight")
    ap.add_argument("--profile-case", action="store_true",
                    help="run two launches of one evaluation (for ncu) and exit")
    ap.add_argument("--profile-k", type=int, default=3000, help="terms (0: trivariate total degree 40)")
    ap.add_argument("--profile-scheme", default="E")
    ap.add_argument("--profile-dtype", default="f64")
    ap.add_argument("--profile-kernel", default="auto", choices=["auto", "ops", "node"])
    ap.add_argument("--profile-ppt", type=int, default=0, help="points per thread (0: automatic)")
    ap.add_argument("--profile-points", type=int, default=0,
                    help="points of the profile case (0: 2^24 univariate, 2^22 trivariate)")
    ap.add_argument("--compose-dtypes", default="modp,f64", help="value types of --workload compose")
    ap.add_argument("--compose-schemes", default="E,B", help="schemes of --workload compose")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default launch shapes)")
    ap.add_argument("--no-configs", action="store_true",
                    help="benchmark line only: skip the other configurations' measurements")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving stream measured beside the benchmark line")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
    elif args.workload == "compose":
        run_compose(args)
    elif args.workload == "compose-accuracy":
        run_compose_accuracy(args)
    elif args.workload == "eval-configs":
        run_eval_config(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "accuracy":
        run_accuracy(args)
    elif args.workload == "staircase":
        run_staircase(args)
    elif args.workload == "hybrid":
        run_hybrid(args)
    elif args.workload == "peaks":
        run_peaks(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "rns":
        run_rns(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
