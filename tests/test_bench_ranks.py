"""The N > 1 host logic of bench.py on two CPU ranks (gloo): rank discovery
from the launcher's environment, the barrier, the max-over-ranks time, the
whole-job value, and the reference arm leaving ranks other than 0 idle."""
import json
import os
import socket
import sys
import time
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, str(ROOT))
    import torch.distributed as dist

    import bench
    got = {"dist": list(bench._dist())}
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    bench._barrier(ws)
    # rank r pretends its timed region took 10 + 5 r ms
    ms = bench._max_over_ranks(10.0 + 5.0 * rank, ws)
    got["max_ms"] = ms
    got["value"] = bench.whole_job_value(1000, ms / 1e3, ws)
    # the reference arm: only rank 0 does work; the others return at once
    if rank != 0:
        class A:
            gpus, steps, warmup = ws, 1, 3
        t0 = time.perf_counter()
        got["ref_rc"] = bench.run_reference(A)
        got["ref_s"] = time.perf_counter() - t0
    bench._barrier(ws)
    dist.destroy_process_group()
    Path(out_dir, f"rank{rank}.json").write_text(json.dumps(got))


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn", join=True)
    r = [json.loads((tmp_path / f"rank{i}.json").read_text()) for i in range(ws)]
    for i in range(ws):
        assert r[i]["dist"] == [ws, i, i]
        assert r[i]["max_ms"] == 15.0  # the slower rank's time, on every rank
        assert r[i]["value"] == pytest.approx(ws * 1000 / 0.015)
    assert r[1]["ref_rc"] == 0 and r[1]["ref_s"] < 1.0


def test_whole_job_value_single():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.whole_job_value(500, 2.0, 1) == 250.0
    assert bench._max_over_ranks(3.5, 1) == 3.5
