#!/usr/bin/env python3
"""Benchmark of the GB300 Projected Adam estimator (one JSON line on rank 0).

Workload: the 401 x 401-cell hydro-mechanical operator (964,806 rows, six
unknowns per cell, 8 inclusions, viscosity 1e18..1e24 Pa s, seed 2), FP64
throughout, one seeded start vector; one step = one kappa_2 estimate =
5000 Projected Adam iterations for sigma_max plus 20000 for sigma_min.
Metric: Projected Adam iterations per second (whole job).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain serial FP64 program under
oracle/) on a bounded sample of the same workload.  Under torchrun with N > 1
every rank runs an independent replica (the estimate does not shard).
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
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "projected_adam_iterations_per_s"
UNIT = "iterations/s"
WORKLOAD = dict(nx=401, ny=401, n_incl=8, eta_lo=1e18, eta_hi=1e24, seed=2)
EST_ITERS = (5000, 20000)  # sigma_max, sigma_min iterations of one kappa_2 estimate
ITERS_MAX, ITERS_MIN = EST_ITERS  # timed per step (overridable for profiling)
HYPER = dict(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12)
START_SEED = 1


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, ws):
    """The slowest rank's time: every rank gets the maximum of x."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank, seconds, ws):
    """Whole-job throughput of ws independent replicas: all ranks' units over
    the slowest rank's time."""
    return ws * units_per_rank / seconds


def flops_per_iteration(n_rows, n_cols, nnz):
    """Algorithmic FP64 flops of one iteration: 2 per entry for each of the
    two products, plus the per-row arithmetic of Algorithm 1 as written
    (gradient 3, moments 7, bias corrections 2, step 4 counting the square
    root and the division as one each, projection 4, update 1, norm 3,
    ||y||^2 and ||x||^2 partials 2 each): 26 per row."""
    return 4 * nnz + 26 * n_cols


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("pa_iter.cu", "pa_device.cuh", "pa_internal.h"):
        h.update((ROOT / "paper_2409_11515_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:16]


def profiled_traffic_per_iteration():
    """DRAM bytes per iteration of k_persistent from the committed ncu summary,
    or None when the kernel source changed since that capture."""
    prof = ROOT / "profiles" / "k_persistent_hydro401.md"
    if not prof.exists():
        return None
    src = dram = None
    for line in prof.read_text().splitlines():
        if line.startswith("kernel source sha256[:16]:"):
            src = line.rsplit(":", 1)[1].strip()
        if line.startswith("dram bytes per iteration:"):
            dram = float(line.split(":", 1)[1].strip())
    return dram if (src == kernel_source_hash() and dram) else None


def bytes_per_iteration(n_rows, n_cols, nnz):
    """Algorithmic bytes of one FP64 iteration: A and A^T read once
    (12 B per entry + 4 B per row pointer) and nine 8-byte vector streams
    per row (x gather, y write, y gather, x read, m r/w, v r/w, x write)."""
    return 2 * (12 * nnz + 4 * (n_rows + 1)) + 72 * n_cols


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2409_11515_gb300 import synth
    A = synth.hydro_operator(WORKLOAD["nx"], WORKLOAD["ny"], n_incl=WORKLOAD["n_incl"],
                             eta_lo=WORKLOAD["eta_lo"], eta_hi=WORKLOAD["eta_hi"],
                             seed=WORKLOAD["seed"])
    oracle.build()
    x0 = oracle.start_vector(A.n_cols, START_SEED)
    sample = 40  # iterations per sigma mode per step: a bounded slice of the estimate
    for _ in range(args.warmup):
        oracle.projected_adam(A, oracle.SIGMA_MAX, 2, x_init=x0, **HYPER)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.projected_adam(A, oracle.SIGMA_MAX, sample, x_init=x0, **HYPER)
        oracle.projected_adam(A, oracle.SIGMA_MIN, sample, x_init=x0, **HYPER)
    dt = time.perf_counter() - t0
    value = 2 * sample * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded hydro-mechanical operator generator)",
        "config": _config(A),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{sample} sigma_max + {sample} sigma_min iterations per step "
                                   "of the 401x401 operator (serial C, -O2, no FMA)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(A):
    return {"workload": "hydro-mechanical 401x401 cells, 6 unknowns/cell, 964806 rows, "
                        "kappa_2 estimate = 5000 sigma_max + 20000 sigma_min iterations",
            "n_rows": int(A.n_rows), "nnz": int(A.nnz), "iters_sigma_max": ITERS_MAX,
            "iters_sigma_min": ITERS_MIN, "precision": "fp64", "k": 1,
            "l2": "working set larger than L2 (A + A^T + 9 vectors of 964806 rows = 231 MB > 129 MB)"}


def cpu_baseline(A, x0):
    import oracle
    oracle.build()
    it = 150
    t0 = time.perf_counter()
    oracle.projected_adam(A, oracle.SIGMA_MAX, it, x_init=x0, **HYPER)
    oracle.projected_adam(A, oracle.SIGMA_MIN, it, x_init=x0, **HYPER)
    dt = time.perf_counter() - t0
    return {"value": 2 * it / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{it} sigma_max + {it} sigma_min iterations of the same operator "
                      "(serial C oracle, one host core)"}


def oracle_iteration_rate(A, iters, x0):
    """Iterations per second of the serial CPU oracle on A: `iters` sigma_max
    and `iters` sigma_min iterations from x0 (one host core)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.projected_adam(A, oracle.SIGMA_MAX, iters, x_init=x0, **HYPER)
    oracle.projected_adam(A, oracle.SIGMA_MIN, iters, x_init=x0, **HYPER)
    return 2 * iters / (time.perf_counter() - t0)


def oracle_estimate_baseline(A, iters):
    """cpu_baseline in kappa_2 estimates/s for one large operator: the oracle's
    iteration rate on a short run, extrapolated to one estimate."""
    import oracle
    rate = oracle_iteration_rate(A, iters, oracle.start_vector(A.n_cols, START_SEED))
    full_T = EST_ITERS[0] + EST_ITERS[1]
    return {"value": rate / full_T, "unit": "estimates/s", "cores": 1, "kind": "oracle",
            "sample": f"{iters} sigma_max + {iters} sigma_min iterations of the same operator "
                      f"(serial C oracle, one host core, {rate:.3g} iterations/s), "
                      f"extrapolated to {EST_ITERS[0]} + {EST_ITERS[1]}"}


def run_ours(args):
    ws, rank, local = _dist()
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2409_11515_gb300 import build, pa, synth
    if rank == 0 or ws == 1:
        build.build()
    _barrier(ws)
    pa.load()
    A = synth.hydro_operator(WORKLOAD["nx"], WORKLOAD["ny"], n_incl=WORKLOAD["n_incl"],
                             eta_lo=WORKLOAD["eta_lo"], eta_hi=WORKLOAD["eta_hi"],
                             seed=WORKLOAD["seed"])
    stream = torch.cuda.Stream()
    tune_rounds = min(args.autotune, 2 * args.warmup)  # all of them inside the warm-up
    h = pa.create(A, stream=stream, autotune=tune_rounds)
    it_per_step = ITERS_MAX + ITERS_MIN

    def step(handle):
        handle.estimate(pa.SIGMA_MAX, ITERS_MAX, seed=START_SEED, **HYPER)
        return handle.estimate(pa.SIGMA_MIN, ITERS_MIN, seed=START_SEED, **HYPER)

    for _ in range(args.warmup):
        r = step(h)
    # ---- device-resident timed region
    sampler = ClockSampler(local)
    launches0 = h.launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    ev0.record(stream)
    for _ in range(args.steps):
        r = step(h)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    _barrier(ws)
    ms = ev0.elapsed_time(ev1)
    ms = _max_over_ranks(ms, ws)
    launches = h.launches() - launches0
    value = whole_job_value(it_per_step * args.steps, ms / 1e3, ws)
    # ---- roofline of the persistent kernel: per-launch time on its own stream
    kms = []
    r_fp64 = None
    for iters, mode in ((ITERS_MAX, pa.SIGMA_MAX), (ITERS_MIN, pa.SIGMA_MIN)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rr = h.estimate(mode, iters, seed=START_SEED, **HYPER)
        e1.record(stream)
        torch.cuda.synchronize()
        kms.append((iters, e0.elapsed_time(e1)))
        r_fp64 = rr
    # ---- mixed precision on the same workload (PA_MIXED): FP32 sigma_max with
    # an FP64 tail, compensated sigma_min; errors against this run's FP64 sigmas
    variants = None
    if not args.no_variants:
        with pa.create(A, stream=stream, precision=pa.MIXED) as hm:
            hm.estimate(pa.SIGMA_MAX, 50, seed=START_SEED, **HYPER)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rm = hm.estimate(pa.SIGMA_MAX, ITERS_MAX, seed=START_SEED, **HYPER)
            e1.record(stream)
            torch.cuda.synchronize()
            t_max = e0.elapsed_time(e1) / 1e3
            it_dd = max(1, ITERS_MIN // 10)
            e0.record(stream)
            rd = hm.estimate(pa.SIGMA_MIN, it_dd, seed=START_SEED, **HYPER)
            e1.record(stream)
            torch.cuda.synchronize()
            t_dd = e0.elapsed_time(e1) / 1e3
        variants = {
            "mixed_sigma_max": {"iterations_per_s": ITERS_MAX / t_max, "iters": ITERS_MAX,
                                "sigma_max": rm["sigma_max"],
                                "rel_err_vs_fp64": abs(rm["sigma_max"] / r_fp64["sigma_max"] - 1),
                                "precision": "FP32 products and Adam state on D_r^-1 A D_c^-1, "
                                             "FP64 norms, last iters/10 in FP64"},
            "compensated_sigma_min": {"iterations_per_s": it_dd / t_dd, "iters": it_dd,
                                      "precision": "FP64 with double-double (Dot2) products"},
        }
    B = bytes_per_iteration(A.n_rows, A.n_cols, A.nnz)
    F = flops_per_iteration(A.n_rows, A.n_cols, A.nnz)
    tot_it = sum(i for i, _ in kms)
    tot_ms = sum(t for _, t in kms)
    achieved = B * tot_it / (tot_ms / 1e3) / 1e9
    achieved_f = F * tot_it / (tot_ms / 1e3) / 1e12
    peak, peak_kind = _peaks()
    clk = clocks.get("sm_mhz") or 2070.0
    # FP64 pipe: 2 FMA lanes per SM per clock (ncu: dfma peak 2/cycle/SM), 152 SMs
    fp64_peak = 2 * 2 * 152 * clk * 1e6 / 1e12
    tpi = profiled_traffic_per_iteration()
    launch_iters = tot_it / len(kms)
    h.destroy()
    # ---- end to end through the C ABI with host buffers
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    _barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with pa.create(A, stream=stream, autotune=tune_rounds) as he:
            he.estimate(pa.SIGMA_MAX, ITERS_MAX, seed=START_SEED, **HYPER)
            re = he.estimate(pa.SIGMA_MIN, ITERS_MIN, seed=START_SEED, **HYPER)
    torch.cuda.synchronize()
    e2e_s = max(_max_over_ranks(time.perf_counter() - t0, ws), 1e-9)
    h2d = A.row_ptr.nbytes + A.col.nbytes + A.val.nbytes + 16 * (ITERS_MAX + ITERS_MIN)
    d2h = 2 * 96 + 4
    if rank == 0:
        traffic = tpi * launch_iters if tpi else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded hydro-mechanical operator generator)",
            "config": dict(_config(A), parallelism=f"replicas{ws}" if ws > 1 else "single_gpu",
                           partition=(f"measured-cost tuner, {tune_rounds} rounds in warm-up"
                                      if tune_rounds > 0 else "fixed cost model")),
            "kappa_estimates_per_s": ws * args.steps / (ms / 1e3),
            "result": {"sigma_max": r["sigma_max"], "sigma_min": r["sigma_min"],
                       "kappa": r["kappa"], "status": r["status"]},
            "roofline": {"bound": "alu", "achieved": achieved_f, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": achieved_f / fp64_peak, "traffic": traffic,
                         "kernel": "k_persistent, FP64 (per-launch CUDA events on its stream)",
                         "peak_source": "FP64 pipe: 2 FMA lanes/SM/clock x 152 SMs x 2 flops "
                                        "x median SM clock under load",
                         "flops_per_iteration": F, "iterations_per_launch": launch_iters,
                         "traffic_source": "ncu dram bytes per iteration x iterations per launch "
                                           "(profiles/k_persistent_hydro401.md)"},
            "roofline_hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "bytes_per_iteration": B,
                             "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json)"},
            "variants_same_workload": variants,
            "clocks": clocks,
            "gpu_launches": launches,
            "e2e": {"value": whole_job_value(it_per_step * e2e_steps, e2e_s, ws), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        }
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(A, _start_vector_host(A.n_cols))
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_batched_workload(args):
    """64 hydro operators with sides drawn from 51..301 (seed 3), 8 restarts
    each, FP64 (or --precision mixed: FP32 sigma_max stage + FP64 tail, Dot2
    sigma_min): vector-iterations per second of pa_estimate_batched (one
    persistent launch sequence per sigma mode, one CUDA graph) against the
    single-vector path looping over the same (matrix, restart) items."""
    if _dist()[0] > 1:
        raise SystemExit("the batched workload runs on one GPU (launch it without torchrun)")
    import torch
    from paper_2409_11515_gb300 import build, pa, synth
    build.build()
    pa.load()
    torch.cuda.set_device(0)
    n_mat, k = 64, 8
    mats = synth.hydro_batch(n_mat, 51, 301, seed=3)
    stream = torch.cuda.Stream()
    mixed = args.precision == "mixed"
    prec = pa.MIXED if mixed else pa.FP64
    # the first handle's autotune picks the restart-block width on a short trial
    hs = [pa.create(A, stream=stream, precision=prec, autotune=1 if i == 0 else 0)
          for i, A in enumerate(mats)]
    rows = sum(A.n_rows for A in mats)
    nnz = sum(A.nnz for A in mats)
    it = (args.iters_max, args.iters_min)
    pa.estimate_batched(hs, pa.BOTH, k, (5, 5), seed=3, **HYPER)  # warm-up
    for _ in range(max(0, args.warmup - 1)):
        pa.estimate_batched(hs, pa.BOTH, k, (5, 5), seed=3, **HYPER)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rb = None
    for _ in range(args.steps):
        rb = pa.estimate_batched(hs, pa.BOTH, k, it, seed=3, **HYPER)
    torch.cuda.synchronize()
    tb = (time.perf_counter() - t0) / args.steps
    vec_its = n_mat * k * (it[0] + it[1])
    # single-vector path over a sample of the same items (every 8th matrix, all restarts)
    sample = list(range(0, n_mat, 8))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in sample:
        for r in range(k):
            hs[i].estimate(pa.SIGMA_MAX, it[0], seed=r, **HYPER)
            hs[i].estimate(pa.SIGMA_MIN, it[1], seed=r, **HYPER)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    frac = sum(mats[i].n_rows for i in sample) / rows
    single_vec_its_per_s = len(sample) * k * (it[0] + it[1]) / ts
    for h in hs:
        h.destroy()
    full_T = EST_ITERS[0] + EST_ITERS[1]
    line = {
        "metric": "kappa2_estimates_per_s (batched, %s)" % ("mixed precision" if mixed else "FP64"),
        "value": n_mat * k / (tb * full_T / (it[0] + it[1])),
        "unit": "estimates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tb * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64", "data": "synthetic (seeded hydro-mechanical operators)",
        "config": {"workload": "64 hydro operators, sides U[51,301] (seed 3), 8 restarts each, "
                               "one persistent SpMM launch per sigma mode in a CUDA graph",
                   "rows_total": rows, "nnz_total": nnz, "k": k,
                   "iters_timed": list(it), "estimate_iters": list(EST_ITERS),
                   "cuda_graph": rb["cuda_graph"]},
        "vector_iterations_per_s": vec_its / tb,
        "single_vector_path": {"vector_iterations_per_s_rowweighted": single_vec_its_per_s,
                               "sample": f"every 8th matrix, all 8 restarts ({frac:.2%} of rows)"},
        "note": "value extrapolates the timed iterations to the 5000 + 20000 of one estimate",
    }
    if not args.no_cpu_baseline:
        import oracle
        cs = list(range(0, n_mat, 16))
        t_cpu = sum(2 * 50 / oracle_iteration_rate(mats[i], 50, oracle.start_vector(mats[i].n_cols, 1))
                    for i in cs)
        # seconds per row-iteration, then one estimate of the batch's average operator
        per_row_it = t_cpu / sum(mats[i].n_rows * 100 for i in cs)
        t_est = per_row_it * (rows / n_mat) * full_T
        line["cpu_baseline"] = {"value": 1.0 / t_est, "unit": "estimates/s", "cores": 1,
                                "kind": "oracle",
                                "sample": "every 16th operator, one restart, 50 + 50 iterations "
                                          "(serial C oracle, one host core), row-weighted and "
                                          "extrapolated to one estimate of the average operator"}
    print(json.dumps(line), flush=True)
    return 0


def _timed(stream, fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    r = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1) / 1e3


def run_mixed1001(args):
    """1001 x 1001 cells (6,012,006 rows, 8 inclusions, viscosity 1e18..1e24,
    seed 4): one kappa_2 estimate (5000 sigma_max + 20000 sigma_min
    iterations) in MIXED precision (pow2 storage equilibration; FP32 sigma_max
    with an FP64 tail, Dot2-compensated FP64 sigma_min) against the same
    estimate in plain FP64 on the same GPU; per-sigma relative differences."""
    if _dist()[0] > 1:
        raise SystemExit("this workload runs on one GPU (launch it without torchrun)")
    import torch
    from paper_2409_11515_gb300 import build, pa, synth
    build.build()
    pa.load()
    torch.cuda.set_device(0)
    A = synth.hydro_operator(1001, n_incl=8, eta_lo=1e18, eta_hi=1e24, seed=4)
    stream = torch.cuda.Stream()
    it_max, it_min = args.iters_max, args.iters_min
    res = {}
    for name, prec in (("fp64", pa.FP64), ("mixed", pa.MIXED)):
        with pa.create(A, stream=stream, precision=prec,
                       autotune=args.autotune if prec == pa.FP64 else 0) as h:
            for _ in range(args.warmup):  # warm-up (and the partition tuner's rounds)
                h.estimate(pa.SIGMA_MAX, 50, seed=START_SEED, **HYPER)
                h.estimate(pa.SIGMA_MIN, 50, seed=START_SEED, **HYPER)
            rM, tM = _timed(stream, lambda: h.estimate(pa.SIGMA_MAX, it_max, seed=START_SEED, **HYPER))
            rm, tm = _timed(stream, lambda: h.estimate(pa.SIGMA_MIN, it_min, seed=START_SEED, **HYPER))
        res[name] = {"sigma_max": rM["sigma_max"], "sigma_min": rm["sigma_min"],
                     "kappa": rM["sigma_max"] / rm["sigma_min"],
                     "sigma_max_iterations_per_s": it_max / tM,
                     "sigma_min_iterations_per_s": it_min / tm,
                     "estimate_s": tM + tm, "status": [rM["status"], rm["status"]]}
    f, m = res["fp64"], res["mixed"]
    line = {
        "metric": "kappa2_estimates_per_s (mixed precision)", "value": 1.0 / m["estimate_s"],
        "unit": "estimates/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": 1e3 * m["estimate_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded hydro-mechanical operator)",
        "config": {"workload": "hydro-mechanical 1001x1001 cells, 6,012,006 rows, pow2 "
                               "equilibration, mixed precision vs FP64",
                   "n_rows": int(A.n_rows), "nnz": int(A.nnz),
                   "iters_sigma_max": it_max, "iters_sigma_min": it_min},
        "fp64_estimates_per_s": 1.0 / f["estimate_s"],
        "rel_diff_vs_fp64": {"sigma_max": abs(m["sigma_max"] / f["sigma_max"] - 1),
                             "sigma_min": abs(m["sigma_min"] / f["sigma_min"] - 1)},
        "runs": res,
        "note": "the comparator is this build's FP64 path (parity-tested against the CPU "
                "oracle); a full-length oracle run at this size takes hours on one core",
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_estimate_baseline(A, 10)
    print(json.dumps(line), flush=True)
    return 0


def run_stress2001(args):
    """2001 x 1001 cells (12,018,006 rows, viscosity 1e16..1e24, k/eta_f
    1e-22..1e-10, seed 5): 32 seeded restarts as SpMM blocks (k = 8 per
    launch, four waves), mixed precision (sigma_max: FP32 stage + FP64 tail;
    sigma_min: Dot2 products) and plain FP64, against the FP64 and mixed-precision
    single-vector paths, each on a short timed run (--iters-max/--iters-min,
    extrapolated to one estimate), plus one full FP64 estimate for kappa_2."""
    if _dist()[0] > 1:
        raise SystemExit("this workload runs on one GPU (launch it without torchrun)")
    import torch
    from paper_2409_11515_gb300 import build, pa, synth
    build.build()
    pa.load()
    torch.cuda.set_device(0)
    A = synth.hydro_operator(2001, 1001, n_incl=8, eta_lo=1e16, eta_hi=1e24, keta_lo=1e-22,
                             keta_hi=1e-10, seed=5)
    stream = torch.cuda.Stream()
    it = (args.iters_max, args.iters_min)
    full_T = EST_ITERS[0] + EST_ITERS[1]
    out = {}
    with pa.create(A, stream=stream, autotune=args.autotune) as h:
        for _ in range(args.warmup):
            h.estimate(pa.SIGMA_MAX, 50, seed=START_SEED, **HYPER)
        r1, t1 = _timed(stream, lambda: (h.estimate(pa.SIGMA_MAX, it[0], seed=START_SEED, **HYPER),
                                         h.estimate(pa.SIGMA_MIN, it[1], seed=START_SEED, **HYPER)))
        out["fp64_k1_vector_iterations_per_s"] = (it[0] + it[1]) / t1
        pa.estimate_batched([h], pa.BOTH, 8, (5, 5), seed=START_SEED, **HYPER)  # warm-up
        rb, tb = _timed(stream, lambda: pa.estimate_batched([h], pa.BOTH, 32, it,
                                                            seed=START_SEED, **HYPER))
        out["fp64_k32_vector_iterations_per_s"] = 32 * (it[0] + it[1]) / tb
        rf, tf = _timed(stream, lambda: (h.estimate(pa.SIGMA_MAX, EST_ITERS[0], seed=START_SEED, **HYPER),
                                         h.estimate(pa.SIGMA_MIN, EST_ITERS[1], seed=START_SEED, **HYPER)))
    with pa.create(A, stream=stream, precision=pa.MIXED) as hm:
        hm.estimate(pa.SIGMA_MAX, 50, seed=START_SEED, **HYPER)
        rmx, tmx = _timed(stream, lambda: hm.estimate(pa.SIGMA_MAX, it[0], seed=START_SEED, **HYPER))
        rmn, tmn = _timed(stream, lambda: hm.estimate(pa.SIGMA_MIN, it[1], seed=START_SEED, **HYPER))
        pa.estimate_batched([hm], pa.BOTH, 8, (5, 5), seed=START_SEED, **HYPER)  # warm-up
        rbm, tbm = _timed(stream, lambda: pa.estimate_batched([hm], pa.BOTH, 32, it,
                                                              seed=START_SEED, **HYPER))
    out["mixed_k1_vector_iterations_per_s"] = (it[0] + it[1]) / (tmx + tmn)
    out["mixed_k32_vector_iterations_per_s"] = 32 * (it[0] + it[1]) / tbm
    kappa = rf[0]["sigma_max"] / rf[1]["sigma_min"]
    est_k32 = 32 * (it[0] + it[1]) / tbm / full_T
    line = {
        "metric": "kappa2_estimates_per_s (32 restarts, mixed-precision SpMM)", "value": est_k32,
        "unit": "estimates/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": 1e3 * tbm, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded hydro-mechanical operator)",
        "config": {"workload": "hydro-mechanical 2001x1001 cells, 12,018,006 rows, viscosity "
                               "contrast 1e8, 32 restarts", "n_rows": int(A.n_rows),
                   "nnz": int(A.nnz), "iters_timed": list(it), "estimate_iters": list(EST_ITERS)},
        "fp64_k1_estimates_per_s": out["fp64_k1_vector_iterations_per_s"] / full_T,
        "fp64_k32_estimates_per_s": out["fp64_k32_vector_iterations_per_s"] / full_T,
        "throughput": out,
        "kappa_fp64_full_estimate": kappa,
        "sigma_fp64": [rf[0]["sigma_max"], rf[1]["sigma_min"]],
        "mixed_short_run_sigmas": [rmx["sigma_max"], rmn["sigma_min"]],
        "batched_sigma_max_spread": [float(rb["sigma_max"].min()), float(rb["sigma_max"].max())],
        "mixed_batched_sigma_max_spread": [float(rbm["sigma_max"].min()), float(rbm["sigma_max"].max())],
        "note": "value and the k=1 figures extrapolate the timed iterations to the 5000 + 20000 "
                "of one estimate; mixed precision: sigma_max FP32 stage + FP64 tail, sigma_min "
                "with Dot2 products (k = 1 and k = 32 alike)",
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_estimate_baseline(A, 10)
    print(json.dumps(line), flush=True)
    return 0


def _lu_factors(A):
    """P A Q = L U from SuperLU (scipy, host): the caller's direct solver."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    from paper_2409_11515_gb300 import synth
    n = A.n_rows
    lu = spl.splu(sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(n, n)).tocsc(),
                  permc_spec="COLAMD")
    out = []
    for T in (lu.L.tocsr(), lu.U.tocsr()):
        T.sort_indices()
        out.append(synth.CSR(T.indptr.astype(np.int32), T.indices.astype(np.int32),
                             T.data.copy(), n, n))
    return (out[0], out[1], np.argsort(lu.perm_r).astype(np.int32),
            np.argsort(lu.perm_c).astype(np.int32))


def run_hydro21(args):
    """The small configuration: the 21 x 21 hydro operator (2,646 rows, 4
    inclusions, seed 1), FP64, 2000 sigma_max + 2000 sigma_min iterations of
    Algorithm 1 per estimate on the thread-block-cluster engine (the grid
    engine's time beside it), and sigma_min through COLAMD LU factors
    (Algorithm 2, 500 iterations) for the kappa_2 the direct route cannot
    reach on this operator."""
    if _dist()[0] > 1:
        raise SystemExit("this workload runs on one GPU (launch it without torchrun)")
    import torch
    from paper_2409_11515_gb300 import build, pa, synth
    build.build()
    pa.load()
    torch.cuda.set_device(0)
    A = synth.hydro_operator(21, seed=1)
    stream = torch.cuda.Stream()
    it = (2000, 2000)
    res = {}
    for name, engine in (("cluster", pa.ENGINE_CLUSTER), ("grid", pa.ENGINE_GRID)):
        with pa.create(A, stream=stream, engine=engine, grid_blocks=16) as h:
            for _ in range(args.warmup):
                h.estimate(pa.BOTH, 50, seed=START_SEED, **HYPER)
            times = []
            for _ in range(args.steps):
                r, dt = _timed(stream, lambda: h.estimate(pa.BOTH, it[0], seed=START_SEED, **HYPER))
                times.append(dt)
            res[name] = {"iterations_per_s": (it[0] + it[1]) * len(times) / sum(times),
                         "us_per_iteration": 1e6 * sum(times) / ((it[0] + it[1]) * len(times)),
                         "sigma_max": r["sigma_max"], "sigma_min_direct": r["sigma_min"]}
    f = _lu_factors(A)
    with pa.create(A, stream=stream) as h:
        h.attach_lu(*f)
        h.estimate(pa.SIGMA_MIN_LU, 20, seed=START_SEED, **HYPER)
        rl, tl = _timed(stream, lambda: h.estimate(pa.BOTH_LU, 500, seed=START_SEED, **HYPER))
    import oracle
    oracle.build()
    x0 = oracle.start_vector(A.n_cols, START_SEED)
    t0 = time.perf_counter()
    oracle.projected_adam(A, oracle.SIGMA_MAX, it[0], x_init=x0, **HYPER)
    oracle.projected_adam(A, oracle.SIGMA_MIN, it[1], x_init=x0, **HYPER)
    t_cpu = time.perf_counter() - t0
    c = res["cluster"]
    line = {
        "metric": METRIC, "value": c["iterations_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * (it[0] + it[1]) / c["iterations_per_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded hydro-mechanical operator)",
        "config": {"workload": "hydro-mechanical 21x21 cells, 2,646 rows, 2000 sigma_max + 2000 "
                               "sigma_min iterations, thread-block-cluster engine (16 CTAs)",
                   "n_rows": int(A.n_rows), "nnz": int(A.nnz), "l2": "working set inside L2"},
        "engines": res,
        "lu_route": {"sigma_max": rl["sigma_max"], "sigma_min": rl["sigma_min"], "kappa": rl["kappa"],
                     "estimate_s": tl, "iters": 500},
        "cpu_baseline": {"value": (it[0] + it[1]) / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "2000 + 2000 iterations of the same operator (serial C oracle)"},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_lu64(args):
    """The paper's full kappa_2 route on many small operators: 64 hydro
    operators with sides drawn from 7..31 cells (seed 6), 8 restarts each;
    sigma_max by Algorithm 1 (FP64 SpMM, 2000 iterations) and sigma_min by
    Algorithm 1 on A^{-1} with Algorithm 2's gradient (given COLAMD LU
    factors, 500 iterations), all items in one pa_estimate_batched call;
    against the single-handle loop and the CPU oracle on the same items."""
    if _dist()[0] > 1:
        raise SystemExit("this workload runs on one GPU (launch it without torchrun)")
    import torch
    from paper_2409_11515_gb300 import build, pa, synth
    build.build()
    pa.load()
    torch.cuda.set_device(0)
    n_mat, k, it = 64, 8, (2000, 500)
    mats = synth.hydro_batch(n_mat, 7, 31, seed=6)
    t0 = time.perf_counter()
    facs = [_lu_factors(A) for A in mats]
    t_factor = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    hs = [pa.create(A, stream=stream) for A in mats]
    for h, f in zip(hs, facs):
        h.attach_lu(*f)
    for _ in range(args.warmup):
        pa.estimate_batched(hs, pa.BOTH_LU, k, (20, 20), seed=3, **HYPER)
    rb, tb = _timed(stream, lambda: pa.estimate_batched(hs, pa.BOTH_LU, k, it, seed=3, **HYPER))
    sample = list(range(0, n_mat, 8))

    def single_loop():
        for i in sample:
            for r in range(2):
                hs[i].estimate(pa.SIGMA_MAX, it[0], seed=r, **HYPER)
                hs[i].estimate(pa.SIGMA_MIN_LU, it[1], seed=r, **HYPER)

    _, ts = _timed(stream, single_loop)
    for h in hs:
        h.destroy()
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for i in sample[:4]:
        x0 = oracle.start_vector(mats[i].n_cols, 1)
        oracle.projected_adam(mats[i], oracle.SIGMA_MAX, it[0], x_init=x0, **HYPER)
        oracle.projected_adam_lu(*facs[i], it[1], x0, **HYPER)
    t_cpu = time.perf_counter() - t0
    rows = [A.n_rows for A in mats]
    kap = rb["kappa"]
    line = {
        "metric": "kappa2_estimates_per_s (LU route, batched)", "value": n_mat * k / tb,
        "unit": "estimates/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": 1e3 * tb, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded hydro-mechanical operators)",
        "config": {"workload": "64 hydro operators, sides U[7,31] (seed 6), 8 restarts each; "
                               "sigma_max 2000 iterations (SpMM), sigma_min 500 iterations on "
                               "A^{-1} through COLAMD LU factors, one CTA per item",
                   "rows_min_max": [min(rows), max(rows)], "k": k, "iters": list(it)},
        "single_handle_estimates_per_s": 2 * len(sample) / ts,
        "cpu_baseline": {"value": len(sample[:4]) / t_cpu, "unit": "estimates/s", "cores": 1,
                         "kind": "oracle",
                         "sample": "4 of the 64 operators, one restart each, same iterations "
                                   "(serial C oracle, one host core)"},
        "kappa_range": [float(np.nanmin(kap)), float(np.nanmax(kap))],
        "item_status_nonzero": int(np.count_nonzero(rb["item_status"])),
        "host_factorisation_s": t_factor,
    }
    print(json.dumps(line), flush=True)
    return 0


def _start_vector_host(n):
    import oracle
    return oracle.start_vector(n, START_SEED)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--autotune", type=int, default=6,
                    help="partition-tuner rounds on the FP64 handle (0 = fixed cost model); "
                         "one per run, so the default 3 warm-up steps (two runs each) hold them")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--no-variants", action="store_true", help="skip the mixed-precision leg")
    ap.add_argument("--workload", choices=["hydro401", "hydro21", "batched", "mixed1001",
                                           "stress2001", "lu64"],
                    default="hydro401",
                    help="hydro401: the benchmark line; hydro21: the small operator (cluster "
                         "engine, LU route); batched: 64 operators x 8 restarts; "
                         "mixed1001: 1001x1001 mixed vs FP64; stress2001: 2001x1001, 32 restarts; "
                         "lu64: 64 small operators, kappa through the LU route")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="batched workload: the handles' precision mode")
    ap.add_argument("--iters-max", type=int, default=None,
                    help="sigma_max iterations per estimate (short runs for profiling); "
                         "default 5000, stress2001 200, batched 500 (timed, then extrapolated)")
    ap.add_argument("--iters-min", type=int, default=None,
                    help="sigma_min iterations; default 20000, stress2001 200, batched 500")
    args = ap.parse_args()
    short = {"stress2001": (200, 200), "batched": (500, 500)}.get(args.workload, EST_ITERS)
    if args.iters_max is None:
        args.iters_max = short[0]
    if args.iters_min is None:
        args.iters_min = short[1]
    globals()["ITERS_MAX"], globals()["ITERS_MIN"] = args.iters_max, args.iters_min
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched_workload(args)
    if args.workload == "mixed1001":
        return run_mixed1001(args)
    if args.workload == "stress2001":
        return run_stress2001(args)
    if args.workload == "lu64":
        return run_lu64(args)
    if args.workload == "hydro21":
        return run_hydro21(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
