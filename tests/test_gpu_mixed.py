"""Mixed precision (PA_MIXED) against the FP64 oracle.

* power-of-two equilibration: bit-exact against the oracle's factors (both
  sides sum the squares in the same order without FMA);
* sigma_max: FP32 products and Adam state on D_r^-1 A D_c^-1, FP64 norms,
  FP64 tail; its sigma_max must match the FP64 oracle's to 1e-6 (the returned
  sigma is ||A x_min|| in FP64, second order in the iterate's error);
* sigma_min: compensated (Dot2) products; the first iterates against the
  oracle's compensated mode within the same rounding-ensemble bar as the FP64
  sigma_min tests.
"""
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


@pytest.mark.parametrize("make", [lambda: synth.hydro_operator(21, seed=1),
                                  lambda: synth.hydro_operator(33, 19, n_incl=8, seed=4),
                                  lambda: synth.random_sparse(900, 7, seed=2, n_cols=700)],
                         ids=["hydro21", "hydro33x19", "rect"])
def test_equilibration_bit_exact(make):
    A = make()
    dr, dc, _ = oracle.equilibrate_pow2(A)
    with pa.create(A, equilibrate=pa.EQ_STORAGE) as h:
        gr, gc = h.get_equilibration()
    assert np.array_equal(gr, dr)
    assert np.array_equal(gc, dc)


@pytest.mark.parametrize("make,T", [(lambda: synth.hydro_operator(21, seed=1), 2000),
                                    (lambda: synth.hydro_operator(17, seed=2), 2000),
                                    (lambda: synth.laplacian_2d(12), 1000),
                                    (lambda: synth.random_sparse(2000, 6, seed=9, diag_boost=3.0), 2000)],
                         ids=["hydro21", "hydro17", "lap2d_12", "random"])
def test_mixed_sigma_max_matches_fp64_oracle(make, T):
    A = make()
    ro = oracle.projected_adam(A, oracle.SIGMA_MAX, T, seed=1, **HYPER)
    with pa.create(A, precision=pa.MIXED) as h:
        r = h.estimate(pa.SIGMA_MAX, T, seed=1, **HYPER)
        x = h.get_vector(pa.SIGMA_MAX)
    assert r["status"] == 0
    assert abs(r["sigma_max"] / ro.sigma - 1) <= 1e-6, (r["sigma_max"], ro.sigma)
    # the returned vector scores the returned sigma (FP64, oracle product)
    assert abs(oracle.sigma(A, x) / r["sigma_max"] - 1) <= 1e-12


def test_mixed_sigma_max_without_tail_and_trace():
    A = synth.hydro_operator(21, seed=1)
    x0 = oracle.start_vector(A.n_cols, 3)
    with pa.create(A, precision=pa.MIXED, fp64_tail=0) as h:
        r = h.run(pa.SIGMA_MAX, 1500, x0, trace_L=True, **HYPER)
    ro = oracle.projected_adam(A, oracle.SIGMA_MAX, 1500, x_init=x0, trace_L=True, **HYPER)
    assert r["iters_run"] == 1500
    assert abs(r["sigma"] / ro.sigma - 1) <= 1e-6
    # the FP32 stage follows the FP64 trajectory to FP32 accuracy at first
    assert np.max(np.abs(r["L_trace"][:20] - ro.L_trace[:20])) <= 1e-4


@pytest.mark.parametrize("name,make", [("hydro21", lambda: synth.hydro_operator(21, seed=1)),
                                       ("lap2d_12", lambda: synth.laplacian_2d(12))])
def test_mixed_sigma_min_dd_iterates(name, make, tmp_path):
    A = make()
    T = 60
    x0 = oracle.start_vector(A.n_cols, 7)
    ref, runs = oracle.rounding_ensemble(A, oracle.SIGMA_MIN, T, x0, tmp_path, flags=oracle.FLAG_DD,
                                         **HYPER)
    spread = np.max([np.linalg.norm(r.x_trace - ref.x_trace, axis=1) for r in runs], axis=0)
    with pa.create(A, precision=pa.MIXED) as h:
        rg = h.run(pa.SIGMA_MIN, T, x0, trace_L=True, n_trace=T, **HYPER)
    err = np.linalg.norm(rg["x_trace"] - ref.x_trace, axis=1)
    quiet = spread <= 1e-12
    assert quiet[:5].all()
    assert np.all(err[quiet] <= 1e-10), np.max(err[quiet])
    assert np.all(err <= np.maximum(1e-10, 100 * spread))
    # the compensated sigma of the returned vector
    assert abs(rg["sigma"] / oracle.sigma(A, rg["x_min"], dd=True) - 1) <= 1e-12


def test_mixed_rejects_quadratic_loss():
    with pytest.raises(pa.PAError) as ei:
        pa.create(synth.laplacian_1d(8), precision=pa.MIXED, loss=pa.LOSS_QUADRATIC)
    assert ei.value.status == -9


# ------------------------------------------------ PA_EQ_TARGET (kappa of A_hat) ---

def _scaled(A):
    dr, dc, vh = oracle.equilibrate_pow2(A)
    return dr, dc, synth.CSR(A.row_ptr, A.col, vh, A.n_rows, A.n_cols)


def test_target_equilibration_holds_the_scaled_matrix():
    """The handle's matrix is A_hat = D_r^-1 A D_c^-1: factors, transpose values and
    products bit-exact / within the product bar of the oracle's A_hat."""
    A = synth.hydro_operator(21, seed=1)
    dr, dc, S = _scaled(A)
    with pa.create(A, equilibrate=pa.EQ_TARGET) as h:
        gr, gc = h.get_equilibration()
        rpt, cit, vat = h.get_transpose()
        x = oracle.start_vector(A.n_cols, 2)
        y = h.spmv(x)
    assert np.array_equal(gr, dr) and np.array_equal(gc, dc)
    order = np.argsort(S.col, kind="stable")
    assert np.array_equal(vat, S.val[order])
    yo = oracle.spmv(S, x)
    absy = oracle.spmv(synth.CSR(S.row_ptr, S.col, np.abs(S.val), S.n_rows, S.n_cols), np.abs(x))
    k = np.diff(S.row_ptr).max()
    assert np.all(np.abs(y - yo) <= 4 * k * 2.0 ** -53 * absy + 1e-300)


@pytest.mark.parametrize("precision", [pa.FP64, pa.MIXED])
def test_target_sigma_max_matches_dense_svd(precision):
    A = synth.hydro_operator(13, seed=1)
    _, _, S = _scaled(A)
    sv = np.linalg.svd(synth.csr_to_dense(S), compute_uv=False)
    with pa.create(A, equilibrate=pa.EQ_TARGET, precision=precision) as h:
        r = h.estimate(pa.SIGMA_MAX, 2000, seed=1, **HYPER)
    assert r["status"] == 0
    # FP64: Algorithm 1's own accuracy after 2000 iterations (the oracle's is
    # 1.5e-10 here); MIXED: the bar of its FP64-oracle comparison
    tol = 1e-8 if precision == pa.FP64 else 1e-6
    assert abs(r["sigma_max"] / sv[0] - 1) <= tol, (r["sigma_max"], sv[0])


def test_target_iterates_match_oracle_on_scaled_matrix():
    A = synth.hydro_operator(21, seed=1)
    _, _, S = _scaled(A)
    T = 100
    x0 = oracle.start_vector(A.n_cols, 7)
    ro = oracle.projected_adam(S, pa.SIGMA_MAX, T, x_init=x0, n_trace=T, trace_L=True, **HYPER)
    with pa.create(A, equilibrate=pa.EQ_TARGET) as h:
        rg = h.run(pa.SIGMA_MAX, T, x0, trace_L=True, n_trace=T, **HYPER)
    assert np.max(np.linalg.norm(rg["x_trace"] - ro.x_trace, axis=1)) <= 1e-10
    assert np.max(np.abs(rg["L_trace"] - ro.L_trace) / np.maximum(1, np.abs(ro.L_trace))) <= 1e-10


def test_unknown_equilibration_rejected():
    with pytest.raises(pa.PAError):
        pa.create(synth.laplacian_2d(5), equilibrate=7)
