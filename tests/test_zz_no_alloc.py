"""pa_sigma_noalloc: the allocation-free sigma = ||A x|| / ||x|| entry point.

It serves callers that cannot allocate device memory where they need the
norm (their memory is held by another allocator, or cudaMalloc's implicit
device synchronisation is not acceptable there).  The tests call it through
the C ABI and compare each result with the CPU oracle's sigma of the same
matrix and vector: on two hydro-mechanical iterates in a row (the calls share
the library's scratch array), on rectangular matrices in both directions, and
on a non-default stream.  They also check that the calls leave the device's
free memory unchanged.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_11515_gb300 import build, pa, synth

pytestmark = pytest.mark.gpu

# Both sides form sqrt(sum y_i^2) / sqrt(sum x_j^2) in FP64 with sums in
# different orders and FMA on the GPU: a few ulp per sum.
REL = 1e-12


def _dev(torch, A):
    dev = torch.device("cuda:0")
    return (torch.from_numpy(A.row_ptr).to(dev), torch.from_numpy(A.col).to(dev),
            torch.from_numpy(A.val).to(dev))


def _free_bytes(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_sigma_noalloc_matches_oracle_twice():
    torch = pytest.importorskip("torch")
    build.build()
    pa.load()
    A = synth.hydro_operator(61, seed=3)
    x0 = oracle.start_vector(A.n_cols, 5)
    with pa.create(A) as h:
        xs = [h.run(pa.SIGMA_MAX, 300, x0)["x_min"], h.run(pa.SIGMA_MIN, 300, x0)["x_min"]]
    dev = torch.device("cuda:0")
    rp, ci, va = _dev(torch, A)
    out = torch.full((1,), math.nan, dtype=torch.float64, device=dev)
    xd = [torch.from_numpy(x).to(dev) for x in xs]
    # the first call on the device looks up the scratch address; after it,
    # two calls in a row must not change the device's free memory
    pa.sigma_noalloc(rp, ci, va, xd[0], out, A.n_rows, A.n_cols)
    free0 = _free_bytes(torch)
    got = []
    for x in xd:  # two calls in a row share the library's scratch
        st = pa.sigma_noalloc(rp, ci, va, x, out, A.n_rows, A.n_cols)
        torch.cuda.synchronize()
        assert st == pa.OK
        got.append(float(out.item()))
    assert _free_bytes(torch) == free0
    for g, x in zip(got, xs):
        want = oracle.sigma(A, x)
        assert abs(g / want - 1) <= REL, (g, want)
    assert got[0] > got[1]


@pytest.mark.parametrize("n_rows,n_cols", [(300, 700), (900, 250)])
def test_sigma_noalloc_rectangular_on_a_stream(n_rows, n_cols):
    torch = pytest.importorskip("torch")
    build.build()
    pa.load()
    A = synth.random_sparse(n_rows, 5, seed=n_rows, n_cols=n_cols)
    x = oracle.start_vector(n_cols, 11) * 3.0  # not unit: ||x|| enters the quotient
    dev = torch.device("cuda:0")
    rp, ci, va = _dev(torch, A)
    xd = torch.from_numpy(x).to(dev)
    out = torch.full((1,), math.nan, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        st = pa.sigma_noalloc(rp, ci, va, xd, out, n_rows, n_cols, stream=s)
    s.synchronize()
    assert st == pa.OK
    M = synth.csr_to_dense(A)
    want = np.linalg.norm(M @ x) / np.linalg.norm(x)
    assert abs(float(out.item()) / want - 1) <= REL
    assert abs(float(out.item()) / oracle.sigma(A, x) - 1) <= REL


def test_sigma_noalloc_rejects_sizes_beyond_its_scratch_and_null_pointers():
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
    L = pa.load()
    st = L.pa_sigma_noalloc(1, 1, rp.data_ptr(), None, va.data_ptr(), x.data_ptr(),
                            out.data_ptr(), None)
    assert st == -1  # PA_ERR_INVALID_ARG
    st = L.pa_sigma_noalloc(1, 1, rp.data_ptr(), ci.data_ptr(), None, x.data_ptr(),
                            out.data_ptr(), None)
    assert st == -1  # PA_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert np.isfinite(out.cpu().numpy()).all()
