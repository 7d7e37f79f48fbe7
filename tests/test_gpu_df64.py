"""Parity of the merged-phase kernel -- in double-float (PA_DF64) and in FP64
(engine MERGED) -- with the CPU oracle, through the C ABI.

PA_DF64 keeps the input in FP64 and recomputes sigma from it in FP64, but
stores the iteration's matrix values and vectors as double-float pairs
(about 48 significant bits) and runs the products and Adam's per-row
arithmetic on the FP32 pipe.  Its bars are the FP64 path's:
  * iterates of Algorithm 1, t <= 100: ||x_t^gpu - x_t^cpu||_2 <= 1e-10 and
    |L_t^gpu - L_t^cpu| <= 1e-10 max(1, |L_t|) for sigma_max;
  * sigma_min iterates: within the oracle's rounding-ensemble bar (1e-10
    where the ensemble stays within 1e-12, else 100x its spread);
  * final kappa within 1e-6 of the closed form;
  * sigma_max within 1e-3 of the oracle's same-seed run on the
    hydro-mechanical operators, sigma_min within 1.5x the ensemble spread.
The merged kernel folds the update of x into the next product; the tests also
cover its fallbacks: iterations that multiply x itself (refresh) and
double-float runs that leave the variant's range and rerun in FP64.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_11515_gb300 import build, pa, synth

from cases import CASES

pytestmark = pytest.mark.gpu

HYPER = dict(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12)
DF = dict(precision=pa.DF64)
MERGED = dict(engine=pa.ENGINE_MERGED)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    pa.load()


def _run(A, mode, T, x0, opt, **kw):
    with pa.create(A, **opt) as h:
        r = h.run(mode, T, x0, **kw, **HYPER)
        r["info"] = h.last_run_info()
    return r


@pytest.mark.parametrize("opt", [DF, MERGED], ids=["df64", "merged_fp64"])
@pytest.mark.parametrize("name", ["hydro21", "hydro13_8incl", "lap2d_12", "random_sparse",
                                  "rect_tall", "rect_wide", "explicit_zeros"])
def test_first_100_iterates_sigma_max(name, opt):
    A = CASES[name]()
    T = 100
    x0 = oracle.start_vector(A.n_cols, 7)
    ro = oracle.projected_adam(A, pa.SIGMA_MAX, T, x_init=x0, n_trace=T, trace_L=True, **HYPER)
    rg = _run(A, pa.SIGMA_MAX, T, x0, opt, trace_L=True, n_trace=T)
    assert rg["info"]["kernel"] == (2 if opt is DF else 1)
    assert rg["status"] == ro.status
    err_x = np.linalg.norm(rg["x_trace"] - ro.x_trace, axis=1)
    err_L = np.abs(rg["L_trace"] - ro.L_trace) / np.maximum(1.0, np.abs(ro.L_trace))
    assert np.max(err_x) <= 1e-10, (np.argmax(err_x), np.max(err_x))
    assert np.max(err_L) <= 1e-10
    assert rg["t_min"] == ro.t_min
    assert abs(rg["sigma"] / ro.sigma - 1) <= 1e-10


@pytest.mark.parametrize("opt", [DF, MERGED], ids=["df64", "merged_fp64"])
@pytest.mark.parametrize("name", ["hydro21", "hydro13_8incl", "lap2d_12", "random_sparse",
                                  "rect_tall"])
def test_first_100_iterates_sigma_min(name, opt, tmp_path):
    """The FP64 path's rounding-ensemble bar (the oracle, its FMA build and
    runs from x_init moved by one ulp in a few entries)."""
    A = CASES[name]()
    T = 100
    x0 = oracle.start_vector(A.n_cols, 7)
    ref, runs = oracle.rounding_ensemble(A, oracle.SIGMA_MIN, T, x0, tmp_path, **HYPER)
    spread = np.max([np.linalg.norm(r.x_trace - ref.x_trace, axis=1) for r in runs], axis=0)
    rg = _run(A, pa.SIGMA_MIN, T, x0, opt, trace_L=True, n_trace=T)
    err = np.linalg.norm(rg["x_trace"] - ref.x_trace, axis=1)
    quiet = spread <= 1e-12
    assert np.all(err[quiet] <= 1e-10), np.max(err[quiet])
    assert np.all(err <= np.maximum(1e-10, 100 * spread)), (err / np.maximum(spread, 1e-300)).max()
    assert quiet[:10].all()


@pytest.mark.parametrize("abl", [pa.ABLATE_NO_TANGENT, pa.ABLATE_NO_NORMALISE,
                                 pa.ABLATE_NO_TANGENT | pa.ABLATE_NO_NORMALISE])
def test_df64_ablation_iterates(abl):
    A = CASES["lap2d_12"]()
    x0 = oracle.start_vector(A.n_cols, 3)
    flags = (oracle.FLAG_NO_TANGENT if abl & pa.ABLATE_NO_TANGENT else 0) | \
            (oracle.FLAG_NO_NORMALISE if abl & pa.ABLATE_NO_NORMALISE else 0)
    ro = oracle.projected_adam(A, oracle.SIGMA_MAX, 50, x_init=x0, flags=flags, n_trace=50, **HYPER)
    rg = _run(A, pa.SIGMA_MAX, 50, x0, dict(DF, ablation=abl), n_trace=50)
    scale = np.maximum(1.0, np.linalg.norm(ro.x_trace, axis=1))
    assert np.max(np.linalg.norm(rg["x_trace"] - ro.x_trace, axis=1) / scale) <= 1e-10


def _lap1d(n):
    h = math.pi / (2 * (n + 1))
    return 1 / math.tan(h) ** 2


@pytest.mark.parametrize("make,kappa", [
    (lambda: synth.laplacian_1d(8), _lap1d(8)),
    (lambda: synth.laplacian_2d(5), _lap1d(5)),
    (lambda: synth.diag_csr([-3.0, 2.5, 0.75, -0.5, 1.25, 2.0, -1.5, 0.6, 1.8, -2.2]), 6.0),
], ids=["lap1d_8", "lap2d_5", "diag"])
def test_df64_closed_form_kappa(make, kappa):
    A = make()
    with pa.create(A, **DF) as h:
        r = h.estimate(pa.BOTH, 3000, seed=1, **HYPER)
        assert h.last_run_info()["kernel"] == 2
    assert r["status"] == 0
    assert abs(r["kappa"] / kappa - 1) <= 1e-6


def test_df64_hydro_sigmas_match_oracle(tmp_path):
    A = synth.hydro_operator(21, seed=1)
    T = 2000
    with pa.create(A, **DF) as h:
        r = h.estimate(pa.BOTH, T, seed=1, **HYPER)
        xm = h.get_vector(pa.SIGMA_MIN)
    ro = oracle.estimate(A, T, T, seed=1, **HYPER)
    assert abs(r["sigma_max"] / ro["sigma_max"] - 1) <= 1e-3
    x0 = oracle.start_vector(A.n_cols, 1)
    _, runs = oracle.rounding_ensemble(A, oracle.SIGMA_MIN, T, x0, tmp_path, n_perturbed=8,
                                       n_entries=16, **HYPER)
    spread = max(abs(rr.sigma / ro["sigma_min"] - 1) for rr in runs)
    assert abs(r["sigma_min"] / ro["sigma_min"] - 1) <= max(1e-3, 1.5 * spread)
    assert r["sigma_min"] <= r["sigma_max"]
    # the returned vector scores the returned sigma (recomputed in FP64)
    assert abs(oracle.sigma(A, xm) / r["sigma_min"] - 1) <= 1e-10


def test_df64_deterministic():
    A = synth.hydro_operator(31, seed=4)
    x0 = oracle.start_vector(A.n_cols, 1)
    with pa.create(A, **DF) as h:
        r1 = h.run(pa.SIGMA_MAX, 200, x0)
        r2 = h.run(pa.SIGMA_MAX, 200, x0)
    assert np.array_equal(r1["x_last"], r2["x_last"])


def test_df64_range_fallbacks():
    # non-zeros spanning more than 2^99: the handle runs the FP64 kernel
    d = np.array([1.0, 2.0 ** -80, 2.0 ** 30, 3.0])
    A = synth.diag_csr(d)
    x0 = oracle.start_vector(4, 2)
    ro = oracle.projected_adam(A, oracle.SIGMA_MAX, 200, x_init=x0, **HYPER)
    with pa.create(A, **DF) as h:
        rg = h.run(pa.SIGMA_MAX, 200, x0, **HYPER)
        assert h.last_run_info()["kernel"] != 2
    assert abs(rg["sigma"] / ro.sigma - 1) <= 1e-12
    # a start on the singular vector of sigma_min = 1e-18 sigma_max: the
    # first ||2^-k A x||^2 lies below 2^-100, the double-float run stops and
    # the run is redone in FP64
    A = synth.diag_csr(np.array([1.0, 0.5, 1e-18, 0.25]))
    x0 = np.array([0.0, 0.0, 1.0, 0.0])
    ro = oracle.projected_adam(A, oracle.SIGMA_MIN, 50, x_init=x0, **HYPER)
    with pa.create(A, **DF) as h:
        rg = h.run(pa.SIGMA_MIN, 50, x0, **HYPER)
        info = h.last_run_info()
    assert info["df_fallbacks"] == 1 and info["kernel"] == 1
    assert rg["status"] == ro.status
    assert abs(rg["sigma"] / ro.sigma - 1) <= 1e-12 and abs(rg["sigma"] / 1e-18 - 1) <= 1e-12


# --------------------------------------------------- full size (C2) ---

@pytest.fixture(scope="module")
def hydro401():
    return synth.hydro_operator(401, n_incl=8, eta_lo=1e18, eta_hi=1e24, seed=2)


@pytest.mark.parametrize("opt", [DF, MERGED], ids=["df64", "merged_fp64"])
@pytest.mark.parametrize("mode", [pa.SIGMA_MAX, pa.SIGMA_MIN])
def test_full_size_first_iterates(hydro401, mode, opt):
    """The 401 x 401 operator (964,806 rows) in the launch configuration the
    benchmark times: L_t for t <= 40 and the iterate x_40.  At this size
    Adam's first steps are mostly radial, so some of these iterations take
    the refresh path (x multiplied itself)."""
    A = hydro401
    T = 40
    x0 = oracle.start_vector(A.n_cols, 1)
    ro = oracle.projected_adam(A, mode, T, x_init=x0, trace_L=True, **HYPER)
    rg = _run(A, mode, T, x0, opt, trace_L=True)
    assert rg["info"]["kernel"] == (2 if opt is DF else 1)
    assert rg["info"]["refreshes"] >= 1
    assert np.linalg.norm(rg["x_last"] - ro.x_last) <= 1e-10
    Lo = ro.L_trace
    assert np.max(np.abs(rg["L_trace"] - Lo) / np.maximum(1, np.abs(Lo))) <= 1e-10


@pytest.mark.parametrize("mode", [pa.SIGMA_MAX, pa.SIGMA_MIN])
def test_df64_6m_rows_first_iterates(mode):
    """The 6,012,006-row operator: L_t for t <= 5 and x_5 against the oracle."""
    A = synth.hydro_operator(1001, n_incl=8, eta_lo=1e18, eta_hi=1e24, seed=4)
    T = 5
    x0 = oracle.start_vector(A.n_cols, 1)
    ro = oracle.projected_adam(A, mode, T, x_init=x0, trace_L=True, **HYPER)
    rg = _run(A, mode, T, x0, DF, trace_L=True)
    assert rg["info"]["kernel"] == 2
    assert np.linalg.norm(rg["x_last"] - ro.x_last) <= 1e-10
    Lo = ro.L_trace
    assert np.max(np.abs(rg["L_trace"] - Lo) / np.maximum(1, np.abs(Lo))) <= 1e-10
