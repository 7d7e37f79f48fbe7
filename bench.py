#!/usr/bin/env python3
"""Benchmark of the GB300 Projected Adam estimator (one JSON line on rank 0).

Workload: the 401 x 401-cell hydro-mechanical operator (964,806 rows, six
unknowns per cell, 8 inclusions, viscosity 1e18..1e24 Pa s, seed 2), FP64
throughout, one seeded start vector; one step = one kappa_2 estimate =
5000 Projected Adam iterations for sigma_max plus 20000 for sigma_min.
Metric: Projected Adam iterations per second (whole job), with the FP64-pipe
and HBM rooflines of the iteration kernel, the relative error of each sigma
against the stored full-length CPU-oracle run, the oracle timed on one host
core and on all host cores (OpenMP build), and an end-to-end figure through
the C ABI with host buffers.

The same line carries bounded runs of the other configurations under
"sub_results" (skip them with --no-sub): the headline workload in PA_DF64
(double-float), the 21 x 21 operator on the cluster engine, 64 operators x 8
restarts in one batched SpMM launch, and the 1001 x 1001 operator in FP64,
PA_DF64 and mixed precision -- each with its roofline, its CPU-oracle
baseline and its errors against the oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload hydro401|hydro21|batched|mixed1001|stress2001|lu64|lu129]

--impl reference times the CPU oracle (the plain serial FP64 program under
oracle/) on a bounded sample of the same workload.  Under torchrun with N > 1
every rank runs an independent replica (the estimate does not shard).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
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
    """HBM copy bandwidth (GB/s) measured on the GB300s, or the
    fallback figure when the measured file is absent."""
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _sm_count():
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp64_peak_tflops(sm_mhz):
    """GB300's FP64 pipe: 2 FMA lanes per SM per clock (ncu's dfma peak), 2
    flops each, times the SM count and the median SM clock under load."""
    return 2 * 2 * _sm_count() * sm_mhz * 1e6 / 1e12


def host_cpu():
    """Core count and CPU model of this host (the oracle's baseline machine)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    if not model:
        try:
            for ln in Path("/proc/cpuinfo").read_text().splitlines():
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model or "unknown", "arch": platform.machine()}


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


KERNEL_SOURCES = {
    "k_persistent": ("pa_iter.cu", "pa_device.cuh", "pa_internal.h"),
    "k_single": ("pa_iter_sp.cu", "pa_device.cuh", "pa_internal.h"),
    "k_merged_df64": ("pa_iter2.cu", "pa_df.cuh", "pa_device.cuh", "pa_internal.h"),
}
TRAFFIC_FILE = ROOT / "profiles" / "dram_traffic.json"


def kernel_source_hash(kernel="k_persistent"):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update((ROOT / "paper_2409_11515_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:16]


def profiled_traffic_per_iteration(kernel="k_persistent", workload="hydro401"):
    """DRAM bytes per iteration of `kernel` on `workload` from the ncu capture
    recorded in profiles/dram_traffic.json, or None when the kernel's sources
    changed since that capture."""
    if not TRAFFIC_FILE.exists():
        return None
    rec = json.loads(TRAFFIC_FILE.read_text()).get(f"{kernel}@{workload}")
    if not rec or rec.get("source_sha16") != kernel_source_hash(kernel):
        return None
    return float(rec["dram_bytes_per_iteration"])


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


def cpu_baseline(A, x0, it=150):
    """The serial oracle on one host core (the contract's baseline) and the
    OpenMP build of the same source on every host core, `it` sigma_max +
    `it` sigma_min iterations of the operator each."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.projected_adam(A, oracle.SIGMA_MAX, it, x_init=x0, **HYPER)
    oracle.projected_adam(A, oracle.SIGMA_MIN, it, x_init=x0, **HYPER)
    dt = time.perf_counter() - t0
    cpu = host_cpu()
    base = {"value": 2 * it / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{it} sigma_max + {it} sigma_min iterations of the same operator "
                      "(serial C oracle, one host core)", "host": cpu}
    try:
        L = oracle.load_openmp()
        with oracle.using(L):
            oracle.projected_adam(A, oracle.SIGMA_MAX, 2, x_init=x0, **HYPER)  # thread start-up
            t0 = time.perf_counter()
            oracle.projected_adam(A, oracle.SIGMA_MAX, it, x_init=x0, **HYPER)
            oracle.projected_adam(A, oracle.SIGMA_MIN, it, x_init=x0, **HYPER)
            dt = time.perf_counter() - t0
        all_cores = {"value": 2 * it / dt, "unit": UNIT,
                     "cores": int(os.environ.get("OMP_NUM_THREADS", cpu["nproc"] or 1)),
                     "kind": "oracle (OpenMP build of the same source, timing only)",
                     "sample": base["sample"].replace("one host core", "all host cores")}
    except (OSError, subprocess.CalledProcessError) as e:
        all_cores = {"unavailable": f"OpenMP build failed: {e}"}
    return base, all_cores


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


def _oracle_run(name):
    """The stored full-length oracle run of a workload (tests/golden), or None."""
    sys.path.insert(0, str(ROOT / "tests" / "golden"))
    try:
        import make_oracle_runs
        return make_oracle_runs.lookup(name)
    except Exception:  # no stored run for the current generator and oracle
        return None


def _rel_err(got, ref, key):
    return None if ref is None else abs(got / ref[key] - 1)


def _timed_events(stream, fn):
    """fn() bracketed by CUDA events on `stream`; (result, seconds)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    r = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1) / 1e3


KAPPA_NOTE = ("sigma_min by the direct route (||A x|| / ||x|| minimised on the sphere): on "
              "these operators it stays far above the true sigma_min, so this kappa is not "
              "kappa_2(A); the paper's route to kappa_2 is Algorithm 2 (PA_SIGMA_MIN_LU)")


def sub_c2_df64(A, stream, it_max, it_min, hbm_peak, ref):
    """The headline workload in PA_DF64 (double-float merged kernel): one full
    estimate timed, its roofline against HBM, its errors against the oracle."""
    from paper_2409_11515_gb300 import pa
    with pa.create(A, stream=stream, precision=pa.DF64, autotune=4) as h:
        for _ in range(2):  # warm-up and two tuner rounds each
            h.estimate(pa.SIGMA_MAX, 500, seed=START_SEED, **HYPER)
            h.estimate(pa.SIGMA_MIN, 500, seed=START_SEED, **HYPER)
        rM, tM = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MAX, it_max, seed=START_SEED, **HYPER))
        infoM = h.last_run_info()
        rm, tm = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MIN, it_min, seed=START_SEED, **HYPER))
        infom = h.last_run_info()
    B = bytes_per_iteration(A.n_rows, A.n_cols, A.nnz)
    its = it_max + it_min
    ach = B * its / (tM + tm) / 1e9
    tpi = profiled_traffic_per_iteration("k_merged_df64")
    return {
        "iterations_per_s": its / (tM + tm), "kappa_estimates_per_s": 1.0 / (tM + tm),
        "precision": "PA_DF64: FP64 input and final sigma; sliced 2^-k A and the vectors as "
                     "double-float pairs (about 48 significant bits), products and Adam on the "
                     "FP32 pipe, reductions in FP64; parity-tested to the FP64 bars",
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                     "frac": ach / hbm_peak, "bytes_per_iteration": B,
                     "traffic": tpi * its / 2 if tpi else None,
                     "kernel": "k_merged<0, true, 2> (per-launch CUDA events)"},
        "result": {"sigma_max": rM["sigma_max"], "sigma_min_direct": rm["sigma_min"],
                   "kappa_direct": rM["sigma_max"] / rm["sigma_min"],
                   "rel_err_vs_oracle": {"sigma_max": _rel_err(rM["sigma_max"], ref, "sigma_max"),
                                         "sigma_min": _rel_err(rm["sigma_min"], ref, "sigma_min")}},
        "run_info": {"sigma_max": infoM, "sigma_min": infom},
    }


def single_pass_bytes(A, info):
    """Bytes of one iteration of the single-pass engine on two bases.
    int32-CSR basis: A read once (12 B per entry + 4 B per row pointer) and
    seven 8-byte vector streams per row (x gather, x read, m r/w, v r/w, x
    write; y stays with the CTA that made it).  Actual basis: what the
    kernel moves -- the sliced copy (12 B per padded entry, 4 B per slice),
    the plan (4 B per slot, 4 B per group lane and per group), the halo
    (8 B written and 8 B read per window column), y and dx through memory
    (16 B each per row) and the seven vector streams."""
    n, nnz = A.n_cols, A.nnz
    csr = 12 * nnz + 4 * (A.n_rows + 1) + 56 * n
    slices = (A.n_rows + 31) // 32
    actual = (12 * info["a_entries"] + 4 * (slices + 1) + 4 * info["plan_slots"]
              + 4 * 33 * info["groups"] + 16 * info["window_cols"] + 32 * n + 56 * n)
    return csr, actual


def sub_c2_single(A, stream, hbm_peak, ref):
    """The headline workload on the single-pass engine (A read once per
    iteration, no transposed copy): one full estimate timed, FP64."""
    from paper_2409_11515_gb300 import pa
    with pa.create(A, stream=stream, engine=pa.ENGINE_SINGLE) as h:
        h.estimate(pa.SIGMA_MAX, 200, seed=START_SEED, **HYPER)  # builds the plans
        rM, tM = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MAX, ITERS_MAX, seed=START_SEED, **HYPER))
        rm, tm = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MIN, ITERS_MIN, seed=START_SEED, **HYPER))
        info = h.single_pass_info()
        run = h.last_run_info()
    its = ITERS_MAX + ITERS_MIN
    t = tM + tm
    csr, actual = single_pass_bytes(A, info)
    two_pass = bytes_per_iteration(A.n_rows, A.n_cols, A.nnz)
    F = flops_per_iteration(A.n_rows, A.n_cols, A.nnz)
    tpi = profiled_traffic_per_iteration("k_single")
    return {
        "engine": "PA_ENGINE_SINGLE (k_single<0>), FP64, "
                  f"{info['grid']} CTAs, {info['window_cols']:,} window columns",
        "iterations_per_s": its / t, "us_per_iteration": 1e6 * t / its,
        "kappa_estimates_per_s": 1.0 / t,
        "roofline": {"bound": "alu", "achieved": F * its / t / 1e12, "unit": "TFLOP/s",
                     "flops_per_iteration": F},
        "roofline_hbm": {"unit": "GB/s", "peak": hbm_peak,
                         "int32_csr_basis": {"bytes_per_iteration": csr,
                                             "achieved": csr * its / t / 1e9,
                                             "frac": csr * its / t / 1e9 / hbm_peak},
                         "actual_basis": {"bytes_per_iteration": actual,
                                          "achieved": actual * its / t / 1e9,
                                          "frac": actual * its / t / 1e9 / hbm_peak},
                         "two_pass_int32_csr_basis_bytes": two_pass,
                         "traffic": tpi * its / 2 if tpi else None},
        "plan": info,
        "result": {"sigma_max": rM["sigma_max"], "sigma_min_direct": rm["sigma_min"],
                   "kappa_direct": rM["sigma_max"] / rm["sigma_min"],
                   "rel_err_vs_oracle": {"sigma_max": _rel_err(rM["sigma_max"], ref, "sigma_max"),
                                         "sigma_min": _rel_err(rm["sigma_min"], ref, "sigma_min")}},
        "run_info": run,
    }


def sub_c2_restarts(A, stream, hbm_peak, k=4, it=(1000, 1000)):
    """The headline operator with k restarts advancing together (one
    pa_estimate_batched call, SpMM blocks), double-float and FP64, a bounded
    run of `it` iterations extrapolated to one estimate per restart; the
    double-float restarts' sigma_max against the FP64 batch's."""
    from paper_2409_11515_gb300 import pa
    out = {}
    res = {}
    B = 2 * (12 * A.nnz + 4 * (A.n_rows + 1)) + 72 * A.n_cols * k  # per batch iteration
    full_T = EST_ITERS[0] + EST_ITERS[1]
    for name, prec in (("df64", pa.DF64), ("fp64", pa.FP64)):
        with pa.create(A, stream=stream, precision=prec) as h:
            pa.estimate_batched([h], pa.BOTH, k, (20, 20), seed=START_SEED, **HYPER)
            r, t = _timed_events(stream, lambda: pa.estimate_batched([h], pa.BOTH, k, it,
                                                                     seed=START_SEED, **HYPER))
        res[name] = r
        its = it[0] + it[1]
        out[name] = {"vector_iterations_per_s": k * its / t,
                     "us_per_vector_iteration": 1e6 * t / (k * its),
                     "kappa_estimates_per_s": k / (t * full_T / its),
                     "roofline": {"bound": "hbm", "achieved": B * its / t / 1e9, "peak": hbm_peak,
                                  "unit": "GB/s", "frac": B * its / t / 1e9 / hbm_peak,
                                  "bytes_per_batch_iteration": B}}
    return {
        "workload": f"hydro 401x401 cells, 964,806 rows, {k} restarts in one pa_estimate_batched "
                    f"call, {it[0]} + {it[1]} iterations timed and extrapolated to one estimate "
                    "per restart",
        "df64": out["df64"], "fp64": out["fp64"],
        "df64_vs_fp64": out["df64"]["vector_iterations_per_s"] / out["fp64"]["vector_iterations_per_s"],
        "sigma_max_rel_diff_df64_vs_fp64": float(
            np.max(np.abs(res["df64"]["sigma_max"] / res["fp64"]["sigma_max"] - 1))),
    }


def sub_c1(stream, steps):
    """C1: the 21 x 21 operator (2,646 rows) on the thread-block-cluster
    engine, 2000 + 2000 iterations per estimate; errors against the oracle's
    same-seed run, which also gives the CPU baseline."""
    import oracle
    from paper_2409_11515_gb300 import pa, synth
    A = synth.hydro_operator(21, seed=1)
    it = 2000
    with pa.create(A, stream=stream, engine=pa.ENGINE_CLUSTER) as h:
        h.estimate(pa.BOTH, 100, seed=START_SEED, **HYPER)
        ts = []
        for _ in range(max(1, steps)):
            r, dt = _timed_events(stream, lambda: h.estimate(pa.BOTH, it, seed=START_SEED, **HYPER))
            ts.append(dt)
        info = h.last_run_info()
    t = sum(ts) / len(ts)
    oracle.build()
    t0 = time.perf_counter()
    ro = oracle.estimate(A, it, it, seed=START_SEED, **HYPER)
    t_cpu = time.perf_counter() - t0
    B = bytes_per_iteration(A.n_rows, A.n_cols, A.nnz)
    F = flops_per_iteration(A.n_rows, A.n_cols, A.nnz)
    return {
        "workload": "hydro 21x21 cells, 2,646 rows, 2000 + 2000 iterations, cluster engine "
                    f"({info['grid']} CTAs)",
        "iterations_per_s": 2 * it / t, "us_per_iteration": 1e6 * t / (2 * it),
        "roofline": {"bound": "alu", "achieved": F * 2 * it / t / 1e12, "unit": "TFLOP/s",
                     "algorithmic_GBps": B * 2 * it / t / 1e9,
                     "note": "working set (0.6 MB) inside L2: latency- and barrier-bound"},
        "result": {"sigma_max": r["sigma_max"], "sigma_min_direct": r["sigma_min"],
                   "rel_err_vs_oracle": {"sigma_max": abs(r["sigma_max"] / ro["sigma_max"] - 1),
                                         "sigma_min": abs(r["sigma_min"] / ro["sigma_min"] - 1)}},
        "cpu_baseline": {"value": 2 * it / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "the same 2000 + 2000 iterations (serial C oracle)"},
    }


def sub_c3(stream, it=(300, 300)):
    """C3: 64 operators (sides U[51, 301], seed 3) x 8 restarts in one
    pa_estimate_batched call (SpMM blocks of k = 8, CUDA graph), a bounded
    run of `it` iterations extrapolated to one estimate; errors of sampled
    items against the oracle from the same start vectors and iterations."""
    import oracle
    from paper_2409_11515_gb300 import pa, synth
    n_mat, k = 64, 8
    mats = synth.hydro_batch(n_mat, 51, 301, seed=3)

    def timed_batch(prec):
        hs = [pa.create(A, stream=stream, precision=prec, autotune=1 if i == 0 else 0)
              for i, A in enumerate(mats)]
        try:
            pa.estimate_batched(hs, pa.BOTH, k, (5, 5), seed=3, **HYPER)
            rb, tb = _timed_events(stream, lambda: pa.estimate_batched(hs, pa.BOTH, k, it, seed=3, **HYPER))
            fb = hs[0].last_run_info()["df_fallbacks"]
        finally:
            for h in hs:
                h.destroy()
        return rb, tb, fb

    rb, tb, _ = timed_batch(pa.FP64)
    rd, td, fbd = timed_batch(pa.DF64)
    full_T = EST_ITERS[0] + EST_ITERS[1]
    K = 8
    B = sum(2 * (12 * A.nnz + 4 * (A.n_rows + 1)) + 72 * A.n_cols * K for A in mats)  # per batch iteration
    F = sum(flops_per_iteration(A.n_rows, A.n_cols, A.nnz) * K for A in mats)
    batch_its = (it[0] + it[1])  # each advances all n_mat x K vectors by one iteration
    hbm_peak, kind = _peaks()
    ach = B * batch_its / tb / 1e9
    oracle.build()
    errs = []
    t_cpu, rows_cpu = 0.0, 0
    for i in (0, 32):
        A = mats[i]
        x0 = oracle.start_vector(A.n_cols, oracle.splitmix64_at(3, i * k + 0))
        t0 = time.perf_counter()
        rM = oracle.projected_adam(A, oracle.SIGMA_MAX, it[0], x_init=x0, **HYPER)
        rm = oracle.projected_adam(A, oracle.SIGMA_MIN, it[1], x_init=x0, **HYPER)
        t_cpu += time.perf_counter() - t0
        rows_cpu += A.n_rows
        errs.append({"item": i, "restart": 0, "rows": int(A.n_rows),
                     "sigma_max": abs(rb["sigma_max"][i, 0] / rM.sigma - 1),
                     "sigma_min": abs(rb["sigma_min"][i, 0] / rm.sigma - 1),
                     "df64_sigma_max": abs(rd["sigma_max"][i, 0] / rM.sigma - 1),
                     "df64_sigma_min": abs(rd["sigma_min"][i, 0] / rm.sigma - 1)})
    rows = sum(A.n_rows for A in mats)
    # the oracle's seconds per row-iteration, scaled to one estimate of every item
    est_cpu = (t_cpu / (rows_cpu * (it[0] + it[1]))) * rows * k * full_T
    return {
        "workload": "64 hydro operators, sides U[51,301] (seed 3), 8 restarts each, one "
                    "persistent SpMM launch per sigma mode (k = 8) in a CUDA graph",
        "rows_total": int(rows), "nnz_total": int(sum(A.nnz for A in mats)),
        "iters_timed": list(it), "cuda_graph": rb["cuda_graph"],
        "vector_iterations_per_s": n_mat * k * batch_its / tb,
        "kappa_estimates_per_s": n_mat * k / (tb * full_T / batch_its),
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                     "frac": ach / hbm_peak, "bytes_per_batch_iteration": B,
                     "fp64_pipe_TFLOPs": F * batch_its / tb / 1e12},
        "rel_err_vs_oracle_sampled": errs,
        "df64": {"engine": "k_batched_df (double-float products and Adam per column, FP64 "
                           "reductions; restart-block width from the tuner's trials)",
                 "vector_iterations_per_s": n_mat * k * batch_its / td,
                 "kappa_estimates_per_s": n_mat * k / (td * full_T / batch_its),
                 "vs_fp64": tb / td, "range_fallbacks": fbd,
                 "roofline": {"bound": "hbm", "achieved": B * batch_its / td / 1e9,
                              "peak": hbm_peak, "unit": "GB/s",
                              "frac": B * batch_its / td / 1e9 / hbm_peak}},
        "cpu_baseline": {"value": n_mat * k / est_cpu, "unit": "estimates/s", "cores": 1,
                         "kind": "oracle",
                         "sample": f"items 0 and 32, restart 0, {it[0]} + {it[1]} iterations "
                                   "(serial C oracle), row-weighted and extrapolated to one "
                                   "estimate of all 512 items"},
        "note": "estimates/s extrapolate the timed iterations to 5000 + 20000 per estimate",
    }


def sub_c4(stream, hbm_peak, dd_iters=1000):
    """C4: the 1001 x 1001 operator (6,012,006 rows): one full FP64 estimate,
    one full PA_DF64 estimate, the MIXED sigma_max (FP32 stage + FP64 tail,
    full length) and a bounded run of the MIXED Dot2 sigma_min; errors of the
    full runs against the stored full-length oracle run."""
    import oracle
    from paper_2409_11515_gb300 import pa, synth
    A = synth.hydro_operator(1001, n_incl=8, eta_lo=1e18, eta_hi=1e24, seed=4)
    ref = _oracle_run("hydro1001")
    B = bytes_per_iteration(A.n_rows, A.n_cols, A.nnz)
    its = EST_ITERS[0] + EST_ITERS[1]
    out = {"workload": "hydro 1001x1001 cells, 6,012,006 rows, 5000 + 20000 iterations",
           "n_rows": int(A.n_rows), "nnz": int(A.nnz), "bytes_per_iteration": B,
           "oracle_reference": "stored full-length run (tests/golden/oracle_runs.json)"
                               if ref else "no stored full-length oracle run for this build"}
    for name, opt in (("fp64", {}), ("df64", dict(precision=pa.DF64))):
        with pa.create(A, stream=stream, **opt) as h:
            h.estimate(pa.SIGMA_MAX, 50, seed=START_SEED, **HYPER)
            rM, tM = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MAX, EST_ITERS[0], seed=START_SEED, **HYPER))
            rm, tm = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MIN, EST_ITERS[1], seed=START_SEED, **HYPER))
            info = h.last_run_info()
        ach = B * its / (tM + tm) / 1e9
        out[name] = {"iterations_per_s": its / (tM + tm), "kappa_estimates_per_s": 1 / (tM + tm),
                     "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                                  "frac": ach / hbm_peak},
                     "sigma_max": rM["sigma_max"], "sigma_min_direct": rm["sigma_min"],
                     "rel_err_vs_oracle": {"sigma_max": _rel_err(rM["sigma_max"], ref, "sigma_max"),
                                           "sigma_min": _rel_err(rm["sigma_min"], ref, "sigma_min")},
                     "kernel": info["kernel"]}
    with pa.create(A, stream=stream, precision=pa.MIXED) as h:
        h.estimate(pa.SIGMA_MAX, 50, seed=START_SEED, **HYPER)
        rM, tM = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MAX, EST_ITERS[0], seed=START_SEED, **HYPER))
        rm, tm = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MIN, dd_iters, seed=START_SEED, **HYPER))
    Bm = 2 * (8 * A.nnz + 4 * (A.n_rows + 1)) + 56 * A.n_cols  # FP32 values/vectors, FP64 m, v
    out["mixed"] = {
        "sigma_max_iterations_per_s": EST_ITERS[0] / tM,
        "sigma_max_roofline": {"bound": "hbm", "achieved": Bm * EST_ITERS[0] / tM / 1e9,
                               "peak": hbm_peak, "unit": "GB/s",
                               "frac": Bm * EST_ITERS[0] / tM / 1e9 / hbm_peak},
        "sigma_max": rM["sigma_max"],
        "sigma_max_rel_err_vs_oracle": _rel_err(rM["sigma_max"], ref, "sigma_max"),
        "dot2_sigma_min_iterations_per_s": dd_iters / tm,
        "kappa_estimates_per_s": 1.0 / (tM + EST_ITERS[1] * tm / dd_iters),
        "note": f"sigma_min (Dot2 products) timed over {dd_iters} iterations and extrapolated"}
    oracle.build()
    t0 = time.perf_counter()
    x0 = oracle.start_vector(A.n_cols, START_SEED)
    oracle.projected_adam(A, oracle.SIGMA_MAX, 5, x_init=x0, **HYPER)
    oracle.projected_adam(A, oracle.SIGMA_MIN, 5, x_init=x0, **HYPER)
    rate = 10 / (time.perf_counter() - t0)
    out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                           "sample": "5 + 5 iterations of the same operator (serial C oracle)",
                           "kappa_estimates_per_s": rate / its}
    return out


def sub_lu129(stream, it_min=100, it_max=2000):
    """The paper's route to kappa_2 at 99,846 rows: the 129 x 129 operator
    (seed 7) with caller-supplied COLAMD LU factors (SuperLU on the host),
    sigma_min by Algorithm 1 on A^{-1} with Algorithm 2's gradient -- the
    factors (27M non-zeros) too large for one CTA's shared memory, so the
    thread-block-cluster kernel runs -- and sigma_max by Algorithm 1; sigma_min's error
    against the oracle's same run, which also gives the CPU baseline."""
    import oracle
    from paper_2409_11515_gb300 import pa, synth
    A = synth.hydro_operator(129, seed=7)
    t0 = time.perf_counter()
    f = _lu_factors(A)
    t_factor = time.perf_counter() - t0
    with pa.create(A, stream=stream) as h:
        h.attach_lu(*f)
        h.estimate(pa.SIGMA_MIN_LU, 5, seed=START_SEED, **HYPER)  # warm-up
        rm, tm = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MIN_LU, it_min, seed=START_SEED, **HYPER))
        info = h.last_run_info()
        rM, tM = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MAX, it_max, seed=START_SEED, **HYPER))
    oracle.build()
    x0 = oracle.start_vector(A.n_cols, START_SEED)
    t0 = time.perf_counter()
    ro = oracle.projected_adam_lu(*f, it_min, x0, **HYPER)
    t_cpu = time.perf_counter() - t0
    nnz_f = int(f[0].nnz + f[1].nnz)
    return {
        "workload": "hydro 129x129 cells, 99,846 rows, COLAMD LU factors "
                    f"({nnz_f:,} non-zeros, about 5,400 levels per triangular system)",
        "kernel": info["kernel"],
        "sigma_min_lu_iterations_per_s": it_min / tm, "ms_per_lu_iteration": 1e3 * tm / it_min,
        "sigma_min_lu": rm["sigma_min"], "sigma_max": rM["sigma_max"],
        "kappa": rM["sigma_max"] / rm["sigma_min"],
        "iters": {"sigma_max": it_max, "sigma_min_lu": it_min},
        "sigma_min_rel_err_vs_oracle": abs(rm["sigma_min"] / ro.sigma_min - 1),
        "roofline": {"bound": "latency",
                     "note": "four triangular solves per iteration, each a chain of about 5,400 "
                             "dependent levels; HBM traffic is not the limit",
                     "factor_bytes_per_iteration": 2 * 12 * nnz_f,
                     "achieved_GBps": 2 * 12 * nnz_f * it_min / tm / 1e9},
        "cpu_baseline": {"value": it_min / t_cpu, "unit": "LU-route iterations/s", "cores": 1,
                         "kind": "oracle", "sample": f"the same {it_min} iterations (serial C oracle)"},
        "host_factorisation_s": t_factor,
    }


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
    df = args.precision == "df64"
    prec = pa.DF64 if df else pa.FP64
    single = args.engine == "single"
    eng = pa.ENGINE_SINGLE if single else pa.ENGINE_AUTO
    h = pa.create(A, stream=stream, autotune=tune_rounds, precision=prec, engine=eng)
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
    for iters, mode in ((ITERS_MAX, pa.SIGMA_MAX), (ITERS_MIN, pa.SIGMA_MIN)):
        _, dt = _timed_events(stream, lambda: h.estimate(mode, iters, seed=START_SEED, **HYPER))
        kms.append((iters, dt * 1e3))
    B = bytes_per_iteration(A.n_rows, A.n_cols, A.nnz)
    F = flops_per_iteration(A.n_rows, A.n_cols, A.nnz)
    tot_it = sum(i for i, _ in kms)
    tot_ms = sum(t for _, t in kms)
    achieved = B * tot_it / (tot_ms / 1e3) / 1e9
    achieved_f = F * tot_it / (tot_ms / 1e3) / 1e12
    peak, peak_kind = _peaks()
    clk = clocks.get("sm_mhz") or 2070.0
    fp64_peak = fp64_peak_tflops(clk)
    ran = h.last_run_info()["kernel"]  # the launch-shape tuner may pick another kernel
    kname = {0: "k_persistent", 1: "k_merged_fp64", 2: "k_merged_df64", 6: "k_single"}.get(ran, "?")
    klabel = {0: "k_persistent<0, 0, 0>, FP64", 1: "k_merged<0, false, 2>, FP64",
              2: "k_merged<0, true, 2>, double-float", 6: "k_single<0>, FP64 single-pass"}.get(ran, "?")
    tpi = profiled_traffic_per_iteration(kname) if kname in KERNEL_SOURCES else None
    launch_iters = tot_it / len(kms)
    choice = h.launch_choice()
    h.destroy()
    ref = _oracle_run("hydro401") if (ITERS_MAX, ITERS_MIN) == EST_ITERS else None
    # ---- the other configurations, each on a bounded sample (rank 0 only)
    subs = None
    if rank == 0 and not args.no_sub and not df and not single:
        subs = {}
        subs["c2_df64"] = sub_c2_df64(A, stream, ITERS_MAX, ITERS_MIN, peak, ref)
        subs["c2_single_pass"] = sub_c2_single(A, stream, peak, ref)
        subs["c2_restarts4"] = sub_c2_restarts(A, stream, peak)
        subs["c1_hydro21_cluster"] = sub_c1(stream, args.steps if args.steps <= 3 else 3)
        subs["c3_batched64"] = sub_c3(stream)
        subs["c4_hydro1001"] = sub_c4(stream, peak)
        subs["lu_hydro129"] = sub_lu129(stream)
    # ---- end to end through the C ABI with host buffers
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    _barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with pa.create(A, stream=stream, autotune=tune_rounds, precision=prec, engine=eng) as he:
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
            "scaling": "weak", "vs_baseline": None, "dtype": "df64 (2xf32)" if df else "f64",
            "data": "synthetic (seeded hydro-mechanical operator generator)",
            "config": dict(_config(A), **({"precision": "PA_DF64"} if df else {})),
            "setup": {"parallelism": f"replicas{ws}" if ws > 1 else "single_gpu",
                      "engine": "single-pass" if single else "auto (three-phase grid kernel)",
                      "partition": (f"measured-cost tuner, {tune_rounds} rounds in warm-up"
                                    if tune_rounds > 0 else "fixed cost model"),
                      "launch_choice": {
                          "kernel": klabel, "ctas": choice["grid"],
                          "source": {0: "not tuned", 1: "timed trials in the warm-up",
                                     2: "cached for this matrix"}[choice["source"]],
                          "trials_ms_40_iterations": [
                              {"kernel": {0: "three-phase", 1: "merged-phase",
                                          6: "single-pass"}.get(k, str(k)),
                               "ctas": g, "ms": round(t, 4)} for k, g, t in choice["trials"]]}},
            "kappa_estimates_per_s": ws * args.steps / (ms / 1e3),
            "result": {"sigma_max": r["sigma_max"], "sigma_min_direct": r["sigma_min"],
                       "kappa_direct": r["kappa"], "kappa_note": KAPPA_NOTE,
                       "status": r["status"],
                       "rel_err_vs_oracle": {"sigma_max": _rel_err(r["sigma_max"], ref, "sigma_max"),
                                             "sigma_min": _rel_err(r["sigma_min"], ref, "sigma_min"),
                                             "reference": "stored full-length oracle run "
                                                          "(tests/golden/oracle_runs.json)"
                                                          if ref else None}},
            "roofline": {"bound": "alu", "achieved": achieved_f, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": achieved_f / fp64_peak, "traffic": traffic,
                         "kernel": klabel + " (per-launch CUDA events on its stream)",
                         "peak_source": f"FP64 pipe: 2 FMA lanes/SM/clock x {_sm_count()} SMs x 2 "
                                        "flops x median SM clock under load (derived)",
                         "flops_per_iteration": F, "iterations_per_launch": launch_iters,
                         "traffic_source": "ncu dram bytes per iteration (profiles/dram_traffic.json) "
                                           "x iterations per launch"},
            "roofline_hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "bytes_per_iteration": B,
                             "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json)"},
            "sub_results": subs,
            "clocks": clocks,
            "gpu_launches": launches,
            "e2e": {"value": whole_job_value(it_per_step * e2e_steps, e2e_s, ws), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        }
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"], line["cpu_baseline_all_cores"] = cpu_baseline(
                A, _start_vector_host(A.n_cols))
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_batched_workload(args):
    """64 hydro operators with sides drawn from 51..301 (seed 3), 8 restarts
    each, FP64 (or --precision mixed: FP32 sigma_max stage + FP64 tail, Dot2
    sigma_min; --precision df64: the double-float SpMM): vector-iterations per second of pa_estimate_batched (one
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
    prec = pa.MIXED if mixed else (pa.DF64 if args.precision == "df64" else pa.FP64)
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
        "metric": "kappa2_estimates_per_s (batched, %s)" % {
            "mixed": "mixed precision", "df64": "double-float"}.get(args.precision, "FP64"),
        "value": n_mat * k / (tb * full_T / (it[0] + it[1])),
        "unit": "estimates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tb * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32+f64", "df64": "df64 (2xf32)"}.get(args.precision, "f64"),
        "data": "synthetic (seeded hydro-mechanical operators)",
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
    single-vector paths and PA_DF64 (k = 1 and the double-float SpMM at k = 32),
    each on a short timed run (--iters-max/--iters-min, extrapolated to one
    estimate), plus one full FP64 estimate for kappa_2."""
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
    # PA_DF64 (double-float iteration held to the FP64 parity bars), k = 1
    with pa.create(A, stream=stream, precision=pa.DF64) as hd:
        hd.estimate(pa.SIGMA_MAX, 50, seed=START_SEED, **HYPER)
        rd, td = _timed(stream, lambda: (hd.estimate(pa.SIGMA_MAX, it[0], seed=START_SEED, **HYPER),
                                         hd.estimate(pa.SIGMA_MIN, it[1], seed=START_SEED, **HYPER)))
        df_info = hd.last_run_info()
        pa.estimate_batched([hd], pa.BOTH, 8, (5, 5), seed=START_SEED, **HYPER)  # warm-up
        rbd, tbd = _timed(stream, lambda: pa.estimate_batched([hd], pa.BOTH, 32, it,
                                                              seed=START_SEED, **HYPER))
    out["df64_k1_vector_iterations_per_s"] = (it[0] + it[1]) / td
    out["df64_k32_vector_iterations_per_s"] = 32 * (it[0] + it[1]) / tbd
    kappa = rf[0]["sigma_max"] / rf[1]["sigma_min"]
    est_k32 = 32 * (it[0] + it[1]) / tbd / full_T
    line = {
        "metric": "kappa2_estimates_per_s (32 restarts, double-float SpMM)", "value": est_k32,
        "unit": "estimates/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": 1e3 * tbd, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "df64 (2xf32)", "data": "synthetic (seeded hydro-mechanical operator)",
        "config": {"workload": "hydro-mechanical 2001x1001 cells, 12,018,006 rows, viscosity "
                               "contrast 1e8, 32 restarts", "n_rows": int(A.n_rows),
                   "nnz": int(A.nnz), "iters_timed": list(it), "estimate_iters": list(EST_ITERS)},
        "mixed_k32_estimates_per_s": 32 * (it[0] + it[1]) / tbm / full_T,
        "fp64_k1_estimates_per_s": out["fp64_k1_vector_iterations_per_s"] / full_T,
        "fp64_k32_estimates_per_s": out["fp64_k32_vector_iterations_per_s"] / full_T,
        "df64_k1_estimates_per_s": out["df64_k1_vector_iterations_per_s"] / full_T,
        "df64_k32_estimates_per_s": out["df64_k32_vector_iterations_per_s"] / full_T,
        "df64_batched_sigma_max_spread": [float(rbd["sigma_max"].min()), float(rbd["sigma_max"].max())],
        "df64_run_info": df_info,
        "df64_short_run_sigmas": [rd[0]["sigma_max"], rd[1]["sigma_min"]],
        "throughput": out,
        "kappa_fp64_full_estimate": kappa,
        "sigma_fp64": [rf[0]["sigma_max"], rf[1]["sigma_min"]],
        "mixed_short_run_sigmas": [rmx["sigma_max"], rmn["sigma_min"]],
        "batched_sigma_max_spread": [float(rb["sigma_max"].min()), float(rb["sigma_max"].max())],
        "mixed_batched_sigma_max_spread": [float(rbm["sigma_max"].min()), float(rbm["sigma_max"].max())],
        "note": "value and the k=1 figures extrapolate the timed iterations to the 5000 + 20000 "
                "of one estimate; value: PA_DF64 handles in pa_estimate_batched (k_batched_df, "
                "restart blocks of the default width K = 4); mixed precision: sigma_max FP32 stage + FP64 tail, "
                "sigma_min with Dot2 products (k = 1 and k = 32 alike)",
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


def run_lu129(args):
    """Algorithm 2's route to sigma_min at 99,846 rows: the 129 x 129 hydro
    operator (seed 7) with caller-supplied COLAMD LU factors (SuperLU on the
    host, 27M non-zeros), Algorithm 1 on A^{-1}; each step one estimate of
    --lu-iters iterations on the thread-block-cluster kernel (engine AUTO),
    the grid kernel's time beside it, and the serial oracle on 5 iterations."""
    if _dist()[0] > 1:
        raise SystemExit("this workload runs on one GPU (launch it without torchrun)")
    import torch
    from paper_2409_11515_gb300 import build, pa, synth
    build.build()
    pa.load()
    torch.cuda.set_device(0)
    A = synth.hydro_operator(129, seed=7)
    f = _lu_factors(A)
    stream = torch.cuda.Stream()
    it = args.lu_iters
    res = {}
    for name, engine in (("auto", pa.ENGINE_AUTO), ("grid", pa.ENGINE_GRID)):
        with pa.create(A, stream=stream, engine=engine) as h:
            h.attach_lu(*f)
            for _ in range(args.warmup):
                h.estimate(pa.SIGMA_MIN_LU, it, seed=START_SEED, **HYPER)
            times = []
            for _ in range(args.steps):
                r, dt = _timed_events(stream, lambda: h.estimate(pa.SIGMA_MIN_LU, it,
                                                                 seed=START_SEED, **HYPER))
                times.append(dt)
            res[name] = {"kernel": h.last_run_info()["kernel"],
                         "ms_per_iteration": 1e3 * sum(times) / (it * len(times)),
                         "sigma_min": r["sigma_min"]}
    import oracle
    oracle.build()
    x0 = oracle.start_vector(A.n_cols, START_SEED)
    t0 = time.perf_counter()
    ro = oracle.projected_adam_lu(*f, 5, x0, **HYPER)
    t_cpu = (time.perf_counter() - t0) / 5
    a = res["auto"]
    nnz_f = int(f[0].nnz + f[1].nnz)
    line = {
        "metric": "sigma_min_lu_iterations_per_s", "value": 1e3 / a["ms_per_iteration"],
        "unit": "iterations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": a["ms_per_iteration"] * it, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded hydro-mechanical operator)",
        "config": {"workload": f"hydro 129x129 cells, 99,846 rows, COLAMD LU factors "
                               f"({nnz_f:,} non-zeros), {it} sigma_min iterations per step "
                               "through Algorithm 2",
                   "n_rows": int(A.n_rows), "factor_nnz": nnz_f, "l2": "factors larger than L2"},
        "engines": res,
        "cpu_baseline": {"value": 1.0 / t_cpu, "unit": "iterations/s", "cores": 1, "kind": "oracle",
                         "sample": "5 iterations of the same operator (serial C oracle)"},
        "oracle_sigma_min_5_iterations": ro.sigma_min,
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
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the bounded runs of the other configurations (C1, C3, C4, DF64)")
    ap.add_argument("--workload", choices=["hydro401", "hydro21", "batched", "mixed1001",
                                           "stress2001", "lu64", "lu129"],
                    default="hydro401",
                    help="hydro401: the benchmark line; hydro21: the small operator (cluster "
                         "engine, LU route); batched: 64 operators x 8 restarts; "
                         "mixed1001: 1001x1001 mixed vs FP64; stress2001: 2001x1001, 32 restarts; "
                         "lu64: 64 small operators, kappa through the LU route; "
                         "lu129: sigma_min through the LU route at 99,846 rows")
    ap.add_argument("--lu-iters", type=int, default=20,
                    help="lu129 only: sigma_min iterations per step")
    ap.add_argument("--precision", choices=["fp64", "mixed", "df64"], default="fp64",
                    help="the handles' precision mode: the default workload takes fp64 "
                         "(the benchmark line) or df64; the batched workload fp64 or mixed")
    ap.add_argument("--engine", choices=["auto", "single"], default="auto",
                    help="hydro401 only: the handle's engine (single: the single-pass "
                         "engine, for profiling it on the benchmark workload)")
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
    if args.workload == "lu129":
        return run_lu129(args)
    if args.workload == "hydro21":
        return run_hydro21(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
