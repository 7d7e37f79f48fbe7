"""The LU route's host analysis (tri_analyse): builds tests/lu_schedule_check.cu
against the library's pa_lu.cu with nvcc (a host program: no GPU needed) and
runs it.  The program replays the step schedule on the CPU, lanes and
butterflies included, and compares it with plain substitution on random
triangular factors (1e-12), checks the staging windows against the padded
arrays, that malformed factors are rejected, and the cluster kernel's form of
each system (lc_build): split by owning CTA, replayed against substitution."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def test_step_schedule_replays_substitution(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if Path("/usr/local/cuda/bin/nvcc").exists() else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "lu_schedule_check"
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", str(ROOT / "include"), "-I", str(ROOT / "paper_2409_11515_gb300" / "csrc"),
           str(ROOT / "tests" / "lu_schedule_check.cu"),
           str(ROOT / "paper_2409_11515_gb300" / "csrc" / "pa_lu.cu"),
           str(ROOT / "paper_2409_11515_gb300" / "csrc" / "pa_lu_cluster.cu"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ALL OK" in r.stdout, r.stdout[-2000:]
