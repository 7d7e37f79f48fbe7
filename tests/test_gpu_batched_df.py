"""pa_estimate_batched with PA_DF64 handles: the double-float SpMM engine.

Item (i, r) is Algorithm 1 on matrix i from the start vector of seed
SplitMix64 output (i * k + r) of the call's seed, as for FP64 batches.  Its
converged sigma_max must match the FP64 oracle's run from the same start
vector to 1e-9 (the FP64 batches' bar), kappa must reach the closed form on
the closed-form matrices (1e-6), reruns are bit-identical, and a batch with a
matrix outside the double-float range runs the FP64 kernel.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_11515_gb300 import build, pa, synth

pytestmark = pytest.mark.gpu
HYPER = dict(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12)
DF = dict(precision=pa.DF64)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    pa.load()


def _x0(n, seed, i, k, r):
    return oracle.start_vector(n, oracle.splitmix64_at(seed, i * k + r))


@pytest.mark.parametrize("k", [1, 3, 8])
def test_df64_batched_sigma_max_matches_oracle(k):
    mats = [synth.hydro_operator(9, seed=1), synth.laplacian_2d(7), synth.hydro_operator(13, 11, seed=2),
            synth.random_sparse(500, 5, seed=3, diag_boost=2.0)]
    hs = [pa.create(A, **DF) for A in mats]
    try:
        T = 1500
        r = pa.estimate_batched(hs, pa.SIGMA_MAX, k, (T, T), seed=9, **HYPER)
        fallbacks = hs[0].last_run_info()["df_fallbacks"]
    finally:
        for h in hs:
            h.destroy()
    assert np.all(r["item_status"] == 0)
    assert fallbacks == 0
    for i, A in enumerate(mats):
        for rr in range(k):
            ro = oracle.projected_adam(A, oracle.SIGMA_MAX, T, x_init=_x0(A.n_cols, 9, i, k, rr),
                                       **HYPER)
            assert abs(r["sigma_max"][i, rr] / ro.sigma - 1) <= 1e-9, (i, rr)


def test_df64_batched_kappa_closed_forms_and_reruns():
    mats = [synth.laplacian_1d(8), synth.laplacian_2d(4), synth.diag_csr([3.0, -0.5, 2.0, 1.5])]
    kappas = [1 / math.tan(math.pi / 18) ** 2, 1 / math.tan(math.pi / 10) ** 2, 6.0]
    hs = [pa.create(A, **DF) for A in mats]
    try:
        r1 = pa.estimate_batched(hs, pa.BOTH, 4, (3000, 3000), seed=2, **HYPER)
        r2 = pa.estimate_batched(hs, pa.BOTH, 4, (3000, 3000), seed=2, **HYPER)
    finally:
        for h in hs:
            h.destroy()
    for i, kap in enumerate(kappas):
        assert np.all(np.abs(r1["kappa"][i] / kap - 1) <= 1e-6), (i, r1["kappa"][i], kap)
    assert np.array_equal(r1["sigma_max"], r2["sigma_max"])
    assert np.array_equal(r1["sigma_min"], r2["sigma_min"])


def test_df64_batched_matches_fp64_batched_on_hydro():
    """Uneven hydro operators, both sigmas after 400 iterations: the
    double-float batch agrees with the FP64 batch to 1e-6 (sigma_max) and
    keeps sigma_min <= sigma_max."""
    mats = [synth.hydro_operator(n, seed=n) for n in (5, 23, 41, 7, 31)]
    out = {}
    for name, opt in (("df", DF), ("fp64", {})):
        hs = [pa.create(A, **opt) for A in mats]
        try:
            out[name] = pa.estimate_batched(hs, pa.BOTH, 2, (400, 400), seed=5, **HYPER)
        finally:
            for h in hs:
                h.destroy()
    a, b = out["df"], out["fp64"]
    assert np.all(a["item_status"] == 0)
    # the double-float kernel ran: its rounding differs from FP64's
    assert not np.array_equal(a["sigma_max"], b["sigma_max"])
    assert np.all(np.abs(a["sigma_max"] / b["sigma_max"] - 1) <= 1e-6)
    assert np.all(a["sigma_min"] <= a["sigma_max"])


def test_df64_batched_out_of_range_matrix_runs_fp64():
    """Non-zeros spanning more than 2^99: the double-float copy is not made,
    so a batch holding that matrix runs the FP64 kernel and gives the FP64
    batch's results bit for bit."""
    mats = [synth.diag_csr(np.array([1.0, 2.0 ** -80, 2.0 ** 30, 3.0])), synth.laplacian_2d(5)]
    out = {}
    for name, opt in (("df", DF), ("fp64", {})):
        hs = [pa.create(A, **opt) for A in mats]
        try:
            out[name] = pa.estimate_batched(hs, pa.BOTH, 3, (500, 500), seed=4, **HYPER)
        finally:
            for h in hs:
                h.destroy()
    assert np.array_equal(out["df"]["sigma_max"], out["fp64"]["sigma_max"])
    assert np.array_equal(out["df"]["sigma_min"], out["fp64"]["sigma_min"])
