"""pa_estimate_batched: many matrices x k restarts in one persistent launch.

Item (i, r) is Algorithm 1 on matrix i from the start vector of seed
SplitMix64 output (i * k + r) of the call's seed; its sigma_max must match
the oracle's run from the same start vector (sigma_max converges: 1e-9),
and kappa must reach the closed form on the closed-form matrices (1e-6).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_11515_gb300 import build, pa, synth

pytestmark = pytest.mark.gpu
HYPER = dict(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    pa.load()


def _x0(n, seed, i, k, r):
    return oracle.start_vector(n, oracle.splitmix64_at(seed, i * k + r))


@pytest.mark.parametrize("k", [1, 3, 8, 10])
def test_batched_sigma_max_matches_oracle(k):
    mats = [synth.hydro_operator(9, seed=1), synth.laplacian_2d(7), synth.hydro_operator(13, 11, seed=2),
            synth.random_sparse(500, 5, seed=3, diag_boost=2.0)]
    hs = [pa.create(A) for A in mats]
    try:
        T = 1500
        r = pa.estimate_batched(hs, pa.SIGMA_MAX, k, (T, T), seed=9, **HYPER)
    finally:
        for h in hs:
            h.destroy()
    assert np.all(r["item_status"] == 0)
    assert r["cuda_graph"]
    for i, A in enumerate(mats):
        for rr in range(k):
            ro = oracle.projected_adam(A, oracle.SIGMA_MAX, T, x_init=_x0(A.n_cols, 9, i, k, rr),
                                       **HYPER)
            assert abs(r["sigma_max"][i, rr] / ro.sigma - 1) <= 1e-9, (i, rr)
    assert np.all(np.isnan(r["sigma_min"]))


def test_batched_kappa_closed_forms_and_single_path():
    mats = [synth.laplacian_1d(8), synth.laplacian_2d(4), synth.diag_csr([3.0, -0.5, 2.0, 1.5])]
    kappas = [1 / math.tan(math.pi / 18) ** 2, 1 / math.tan(math.pi / 10) ** 2, 6.0]
    hs = [pa.create(A) for A in mats]
    try:
        r = pa.estimate_batched(hs, pa.BOTH, 4, (3000, 3000), seed=2, **HYPER)
        # the batched item equals the single-vector run from the same start vector
        x0 = _x0(mats[1].n_cols, 2, 1, 4, 3)
        single = hs[1].run(pa.SIGMA_MAX, 3000, x0, **HYPER)
    finally:
        for h in hs:
            h.destroy()
    for i, kap in enumerate(kappas):
        assert np.all(np.abs(r["kappa"][i] / kap - 1) <= 1e-6), (i, r["kappa"][i], kap)
    assert abs(r["sigma_max"][1, 3] / single["sigma"] - 1) <= 1e-12


def test_batched_uneven_sizes_deterministic():
    mats = [synth.hydro_operator(n, seed=n) for n in (5, 23, 41, 7, 31)]
    hs = [pa.create(A) for A in mats]
    try:
        r1 = pa.estimate_batched(hs, pa.BOTH, 2, (400, 400), seed=5, **HYPER)
        r2 = pa.estimate_batched(hs, pa.BOTH, 2, (400, 400), seed=5, **HYPER)
    finally:
        for h in hs:
            h.destroy()
    assert np.array_equal(r1["sigma_max"], r2["sigma_max"])
    assert np.array_equal(r1["sigma_min"], r2["sigma_min"])
    assert np.all(r1["sigma_min"] <= r1["sigma_max"])
    for i, A in enumerate(mats):  # sigma_max after 400 iterations: within 1e-6 of the oracle
        ro = oracle.projected_adam(A, oracle.SIGMA_MAX, 400, x_init=_x0(A.n_cols, 5, i, 2, 0), **HYPER)
        assert abs(r1["sigma_max"][i, 0] / ro.sigma - 1) <= 1e-6


def test_batched_errors():
    with pa.create(synth.random_sparse(30, 3, seed=1, n_cols=40)) as h:
        with pytest.raises(pa.PAError) as ei:
            pa.estimate_batched([h], pa.SIGMA_MIN, 2, (10, 10))
        assert ei.value.status == -3
    with pa.create(synth.laplacian_1d(8), precision=pa.MIXED) as hm, pa.create(synth.laplacian_1d(9)) as hf:
        with pytest.raises(pa.PAError) as ei:  # one precision mode per batch
            pa.estimate_batched([hm, hf], pa.SIGMA_MAX, 2, (10, 10))
        assert ei.value.status == -1


def test_batched_autotuned_width_keeps_results():
    """With autotune on the first handle the engine times restart blocks of
    8, 4 and 2 vectors on a short trial and keeps the fastest; every item
    still matches the untuned batch (only the reduction order may differ)."""
    mats = [synth.hydro_operator(9, seed=1), synth.hydro_operator(13, 11, seed=2),
            synth.random_sparse(500, 5, seed=3, diag_boost=2.0)]
    k, T = 8, 1500
    hs = [pa.create(A, autotune=1 if i == 0 else 0) for i, A in enumerate(mats)]
    hd = [pa.create(A) for A in mats]
    try:
        rt = pa.estimate_batched(hs, pa.BOTH, k, (T, T), seed=4, **HYPER)
        rt2 = pa.estimate_batched(hs, pa.BOTH, k, (T, T), seed=4, **HYPER)  # cached width
        rd = pa.estimate_batched(hd, pa.BOTH, k, (T, T), seed=4, **HYPER)
    finally:
        for h in hs + hd:
            h.destroy()
    assert rt["status"] == 0 and rd["status"] == 0
    assert np.array_equal(rt["sigma_max"], rt2["sigma_max"])
    assert np.max(np.abs(rt["sigma_max"] / rd["sigma_max"] - 1)) <= 1e-9


# MIXED handles: sigma_max runs the FP32 SpMM stage (FP32 products and Adam
# state on the power-of-two-equilibrated matrix) and an FP64 tail; each item
# must match the FP64 oracle from its start vector to the single-vector MIXED
# bar (1e-6, both converged), and sigma_min (FP64) the closed form.
@pytest.mark.parametrize("k", [1, 3, 8])
def test_batched_mixed_sigma_max_matches_fp64_oracle(k):
    mats = [synth.hydro_operator(9, seed=1), synth.laplacian_2d(7), synth.hydro_operator(13, 11, seed=2),
            synth.random_sparse(500, 5, seed=3, diag_boost=2.0)]
    hs = [pa.create(A, precision=pa.MIXED) for A in mats]
    try:
        T = 2000
        r = pa.estimate_batched(hs, pa.SIGMA_MAX, k, (T, T), seed=9, **HYPER)
        r2 = pa.estimate_batched(hs, pa.SIGMA_MAX, k, (T, T), seed=9, **HYPER)
    finally:
        for h in hs:
            h.destroy()
    assert np.all(r["item_status"] == 0)
    assert np.array_equal(r["sigma_max"], r2["sigma_max"])  # bit-reproducible
    for i, A in enumerate(mats):
        for rr in range(k):
            ro = oracle.projected_adam(A, oracle.SIGMA_MAX, T, x_init=_x0(A.n_cols, 9, i, k, rr),
                                       **HYPER)
            assert abs(r["sigma_max"][i, rr] / ro.sigma - 1) <= 1e-6, (i, rr, r["sigma_max"][i, rr], ro.sigma)


def test_batched_mixed_fp32_stage_only_and_kappa():
    mats = [synth.laplacian_1d(8), synth.laplacian_2d(4), synth.hydro_operator(11, seed=4)]
    hs = [pa.create(A, precision=pa.MIXED, fp64_tail=0) for A in mats]
    try:
        T = 2000
        r = pa.estimate_batched(hs, pa.BOTH, 2, (T, 3000), seed=4, **HYPER)
    finally:
        for h in hs:
            h.destroy()
    assert np.all(r["item_status"] == 0)
    for i, A in enumerate(mats):  # the FP32 stage alone reaches the FP64 oracle's sigma_max
        for rr in range(2):
            ro = oracle.projected_adam(A, oracle.SIGMA_MAX, T, x_init=_x0(A.n_cols, 4, i, 2, rr), **HYPER)
            assert abs(r["sigma_max"][i, rr] / ro.sigma - 1) <= 1e-6, (i, rr)
    kappas = [1 / math.tan(math.pi / 18) ** 2, 1 / math.tan(math.pi / 10) ** 2]
    for i, kap in enumerate(kappas):
        assert np.all(np.abs(r["kappa"][i] / kap - 1) <= 1e-6), (i, r["kappa"][i], kap)


def test_batched_mixed_sigma_min_dot2_matches_oracle():
    # a MIXED batch runs sigma_min with Dot2 products (the oracle's FLAG_DD
    # reading of them); on matrices where sigma_min converges the batched
    # items reach the oracle's value from the same start vectors
    mats = [synth.laplacian_1d(12), synth.laplacian_2d(6)]
    hs = [pa.create(A, precision=pa.MIXED) for A in mats]
    try:
        T = 3000
        r = pa.estimate_batched(hs, pa.SIGMA_MIN, 2, (T, T), seed=7, **HYPER)
    finally:
        for h in hs:
            h.destroy()
    assert np.all(r["item_status"] == 0)
    assert np.all(np.isnan(r["sigma_max"]))
    for i, A in enumerate(mats):
        for rr in range(2):
            ro = oracle.projected_adam(A, oracle.SIGMA_MIN, T, x_init=_x0(A.n_cols, 7, i, 2, rr),
                                       flags=oracle.FLAG_DD, **HYPER)
            assert abs(r["sigma_min"][i, rr] / ro.sigma - 1) <= 1e-6, (i, rr, r["sigma_min"][i, rr], ro.sigma)


def test_batched_mixed_with_no_fp32_iterations():
    # fp64_tail = iters: the FP32 stage runs no iteration, so its tracked
    # minimiser must be x_init and the FP64 tail decides; iters = 0 scores
    # x_init itself (through its FP32 copy: 1e-6)
    mats = [synth.laplacian_2d(7), synth.hydro_operator(9, seed=1)]
    T = 1500
    hs = [pa.create(A, precision=pa.MIXED, fp64_tail=T) for A in mats]
    try:
        r = pa.estimate_batched(hs, pa.SIGMA_MAX, 2, (T, T), seed=5, **HYPER)
        r0 = pa.estimate_batched(hs, pa.SIGMA_MAX, 2, (0, 0), seed=5, **HYPER)
    finally:
        for h in hs:
            h.destroy()
    assert np.all(r["item_status"] == 0) and np.all(r0["item_status"] == 0)
    for i, A in enumerate(mats):
        for rr in range(2):
            x0 = _x0(A.n_cols, 5, i, 2, rr)
            ro = oracle.projected_adam(A, oracle.SIGMA_MAX, T, x_init=x0, **HYPER)
            assert abs(r["sigma_max"][i, rr] / ro.sigma - 1) <= 1e-6, (i, rr)
            assert abs(r0["sigma_max"][i, rr] / oracle.sigma(A, x0) - 1) <= 1e-6, (i, rr)
