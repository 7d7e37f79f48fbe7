"""Write oracle_runs.json: full-length CPU-oracle runs of the benchmark workloads.

Each entry is one kappa_2 estimate of Algorithm 1 (sigma_max and sigma_min
from the same seeded start vector) computed by the plain serial FP64 oracle
(oracle/pa_oracle.c) alone -- no CUDA code is involved.  The benchmark reads
them to state each timed run's relative error per sigma against the oracle.

Entries are keyed by a hash of everything the result depends on: the
generator arguments, the iteration counts, the hyperparameters, the start
seed and the oracle's source text.  A key that no longer matches (a changed
generator, oracle or workload) simply goes unused.

    python tests/golden/make_oracle_runs.py [workload ...]

Workloads: hydro401 (964,806 rows, 5000 + 20000 iterations: about 7 minutes
on one core) and hydro1001 (6,012,006 rows: about an hour).  The runs are
made on whatever host runs the script; sigma_min of these operators is not
reproducible to better than tens of percent under round-off (the oracle's own
rounding ensemble), so a different host's libm may give another member of
that ensemble.
"""
from __future__ import annotations

import hashlib
import json
import platform
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2409_11515_gb300 import synth  # noqa: E402

OUT = Path(__file__).resolve().parent / "oracle_runs.json"
HYPER = dict(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12)

WORKLOADS = {
    "hydro401": dict(gen=dict(nx=401, ny=401, n_incl=8, eta_lo=1e18, eta_hi=1e24, seed=2),
                     iters=(5000, 20000), start_seed=1),
    "hydro1001": dict(gen=dict(nx=1001, ny=1001, n_incl=8, eta_lo=1e18, eta_hi=1e24, seed=4),
                      iters=(5000, 20000), start_seed=1),
}


def key(name: str) -> str:
    w = WORKLOADS[name]
    h = hashlib.sha256()
    h.update(json.dumps({"gen": w["gen"], "iters": w["iters"], "seed": w["start_seed"],
                         "hyper": HYPER}, sort_keys=True).encode())
    h.update(oracle.source_text().encode())
    return f"{name}:{h.hexdigest()[:16]}"


def operator(name: str):
    g = dict(WORKLOADS[name]["gen"])
    return synth.hydro_operator(g.pop("nx"), g.pop("ny"), **g)


def run(name: str) -> dict:
    w = WORKLOADS[name]
    A = operator(name)
    t0 = time.time()
    r = oracle.estimate(A, w["iters"][0], w["iters"][1], seed=w["start_seed"], **HYPER)
    return {"workload": name, "n_rows": int(A.n_rows), "nnz": int(A.nnz),
            "iters": list(w["iters"]), "start_seed": w["start_seed"], "hyper": HYPER,
            "sigma_max": r["sigma_max"], "sigma_min": r["sigma_min"], "kappa": r["kappa"],
            "t_min_max": r["max"].t_min, "t_min_min": r["min"].t_min,
            "status": [r["status_max"], r["status_min"]],
            "seconds": round(time.time() - t0, 1),
            "host": f"{platform.machine()} {platform.processor() or ''}".strip()}


def load() -> dict:
    return json.loads(OUT.read_text()) if OUT.exists() else {}


def lookup(name: str):
    """The stored run of `name` for the current generator and oracle, or None."""
    return load().get(key(name))


def main(names):
    oracle.build()
    for name in names:
        r = run(name)
        data = load()  # re-read: another invocation may have added its run meanwhile
        data[key(name)] = r
        OUT.write_text(json.dumps(data, indent=1, sort_keys=True) + "\n")
        print(name, r, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
