"""pa_sigma_noalloc: the allocation-free sigma = ||A x|| / ||x|| entry point.

It serves callers that cannot allocate device memory where they need the
norm (their memory is held by another allocator, or cudaMalloc's implicit
device synchronisation is not acceptable there).  The test calls it through
the C ABI on two vectors in a row and compares each result with the sigma
that pa_run (the existing entry point, which allocates its buffers) reports
for the same vector.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_11515_gb300 import build, pa, synth

pytestmark = pytest.mark.gpu


def test_sigma_noalloc_matches_pa_run_twice():
    torch = pytest.importorskip("torch")
    build.build()
    pa.load()
    A = synth.hydro_operator(61, seed=3)
    x0 = oracle.start_vector(A.n_cols, 5)
    with pa.create(A) as h:
        r_max = h.run(pa.SIGMA_MAX, 300, x0)
        r_min = h.run(pa.SIGMA_MIN, 300, x0)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col).to(dev)
    va = torch.from_numpy(A.val).to(dev)
    out = torch.full((1,), math.nan, dtype=torch.float64, device=dev)
    for r in (r_max, r_min):  # two calls in a row share the library's scratch
        x = torch.from_numpy(r["x_min"]).to(dev)
        torch.cuda.synchronize()
        st = pa.sigma_noalloc(rp, ci, va, x, out, A.n_rows, A.n_cols)
        torch.cuda.synchronize()
        assert st == pa.OK
        got = float(out.item())
        assert abs(got / r["sigma"] - 1) <= 1e-12, (got, r["sigma"])
    assert r_max["sigma"] > r_min["sigma"]


def test_sigma_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    build.build()
    pa.load()
    dev = torch.device("cuda:0")
    rp = torch.zeros(2, dtype=torch.int32, device=dev)
    ci = torch.zeros(1, dtype=torch.int32, device=dev)
    va = torch.zeros(1, dtype=torch.float64, device=dev)
    x = torch.zeros(1, dtype=torch.float64, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(pa.PAError) as ei:
        pa.sigma_noalloc(rp, ci, va, x, out, 2_097_153, 1)
    assert ei.value.status == -1 and "limit" in str(ei.value)
    assert np.isfinite(out.cpu().numpy()).all()
