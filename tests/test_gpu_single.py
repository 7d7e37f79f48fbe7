"""Parity of the single-pass engine (A read once per iteration, no transposed
copy; Eq. nabla_loss's A^T A x from per-CTA window plans) with the CPU oracle.

Bars, as for the three-phase kernel:
  * z = A^T (A x) per entry: |gpu - oracle| <= sum_i |a_ij| e_i + 4 k' u sum_i |a_ij y_i|
    with e_i = 4 k u sum_j |a_ij x_j| the bound on y_i (k, k': entries per row
    of A and of A^T; the sides differ in FMA use and in the order of the
    column sums, which here run over CTA windows);
  * iterates of Algorithm 1, t <= 100: ||x_t^gpu - x_t^cpu||_2 <= 1e-10 and
    |L_t^gpu - L_t^cpu| <= 1e-10 max(1, |L_t|) (sigma_min: the rounding-ensemble
    bar of the three-phase kernel's tests);
  * reruns bit-identical (every sum has a fixed order).
"""
import numpy as np
import pytest

import oracle
from paper_2409_11515_gb300 import build, pa, synth

from cases import CASES

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
HYPER = dict(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12)
SINGLE = dict(engine=pa.ENGINE_SINGLE)
SQUARE = ["explicit_zeros", "hydro21", "hydro13_8incl", "lap2d_12", "random_sparse"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    pa.load()


def _abs(A):
    return synth.CSR(A.row_ptr, A.col, np.abs(A.val), A.n_rows, A.n_cols)


def _ata_bound(A, x, y):
    """Per-entry bound on |z_gpu - A^T y| for z_gpu = A^T (A x)_gpu, y = A x (oracle)."""
    k = max(int(np.diff(A.row_ptr).max()), 1)
    kt = max(int(np.bincount(A.col, minlength=A.n_cols).max()), 1)
    e_y = 4 * k * U * oracle.spmv(_abs(A), np.abs(x))
    return oracle.spmv_t(_abs(A), e_y) + 4 * kt * U * oracle.spmv_t(_abs(A), np.abs(y)) + 1e-300


@pytest.mark.parametrize("grid", [0, 7])
@pytest.mark.parametrize("name", SQUARE)
def test_ata_product_matches_oracle(name, grid):
    A = CASES[name]()
    x = np.random.default_rng(2).standard_normal(A.n_cols)
    with pa.create(A, grid_blocks=grid, **SINGLE) as h:
        z = h.spmv_ata(x)
        info = h.single_pass_info()
    y = oracle.spmv(A, x)
    zo = oracle.spmv_t(A, y)
    assert np.all(np.abs(z - zo) <= _ata_bound(A, x, y))
    # one plan entry per stored non-zero
    assert info["plan_entries"] == int(np.count_nonzero(A.val))
    if grid:  # at most one CTA per 32-row slice
        assert info["grid"] == min(grid, (A.n_rows + 31) // 32)


def _iterate_parity(A, mode, T=100, seed=7, **opt):
    x0 = oracle.start_vector(A.n_cols, seed)
    ro = oracle.projected_adam(A, mode, T, x_init=x0, n_trace=T, trace_L=True,
                               loss=opt.get("loss", pa.LOSS_LOGRATIO), **HYPER)
    with pa.create(A, **SINGLE, **opt) as h:
        rg = h.run(mode, T, x0, trace_L=True, n_trace=T, **HYPER)
        assert h.last_run_info()["kernel"] == 6
    assert rg["status"] == ro.status
    err_x = np.linalg.norm(rg["x_trace"] - ro.x_trace, axis=1)
    err_L = np.abs(rg["L_trace"] - ro.L_trace) / np.maximum(1.0, np.abs(ro.L_trace))
    return rg, ro, err_x, err_L


@pytest.mark.parametrize("grid", [0, 7])
@pytest.mark.parametrize("name", SQUARE)
def test_first_100_iterates_sigma_max(name, grid):
    A = CASES[name]()
    rg, ro, err_x, err_L = _iterate_parity(A, pa.SIGMA_MAX, grid_blocks=grid)
    assert np.max(err_x) <= 1e-10, (np.argmax(err_x), np.max(err_x))
    assert np.max(err_L) <= 1e-10
    assert rg["t_min"] == ro.t_min
    assert abs(rg["sigma"] / ro.sigma - 1) <= 1e-10


@pytest.mark.parametrize("name", ["hydro21", "hydro13_8incl", "lap2d_12", "random_sparse"])
def test_first_100_iterates_sigma_min(name, tmp_path):
    """The three-phase kernel's sigma_min bar: 1e-10 while the oracle's
    rounding ensemble stays within 1e-12 of the oracle, 100x its spread after."""
    A = CASES[name]()
    T = 100
    x0 = oracle.start_vector(A.n_cols, 7)
    ref, runs = oracle.rounding_ensemble(A, oracle.SIGMA_MIN, T, x0, tmp_path, **HYPER)
    spread = np.max([np.linalg.norm(r.x_trace - ref.x_trace, axis=1) for r in runs], axis=0)
    with pa.create(A, grid_blocks=5, **SINGLE) as h:
        rg = h.run(pa.SIGMA_MIN, T, x0, trace_L=True, n_trace=T, **HYPER)
    err = np.linalg.norm(rg["x_trace"] - ref.x_trace, axis=1)
    quiet = spread <= 1e-12
    assert np.all(err[quiet] <= 1e-10), np.max(err[quiet])
    assert np.all(err <= np.maximum(1e-10, 100 * spread))
    assert quiet[:10].all()


@pytest.mark.parametrize("mode", [pa.SIGMA_MAX, pa.SIGMA_MIN])
def test_quadratic_loss_iterates(mode):
    A = CASES["hydro21"]()
    rg, ro, err_x, err_L = _iterate_parity(A, mode, loss=pa.LOSS_QUADRATIC, grid_blocks=4)
    assert np.max(err_x) <= 1e-10
    assert np.max(err_L) <= 1e-10


@pytest.mark.parametrize("abl", [pa.ABLATE_NO_TANGENT, pa.ABLATE_NO_NORMALISE])
def test_ablation_iterates(abl):
    A = CASES["lap2d_12"]()
    x0 = oracle.start_vector(A.n_cols, 3)
    flags = oracle.FLAG_NO_TANGENT if abl == pa.ABLATE_NO_TANGENT else oracle.FLAG_NO_NORMALISE
    ro = oracle.projected_adam(A, oracle.SIGMA_MAX, 50, x_init=x0, flags=flags, n_trace=50, **HYPER)
    with pa.create(A, ablation=abl, grid_blocks=3, **SINGLE) as h:
        rg = h.run(pa.SIGMA_MAX, 50, x0, n_trace=50, **HYPER)
    scale = np.maximum(1.0, np.linalg.norm(ro.x_trace, axis=1))
    assert np.max(np.linalg.norm(rg["x_trace"] - ro.x_trace, axis=1) / scale) <= 1e-10


def test_reruns_bit_identical():
    A = synth.hydro_operator(31, seed=4)
    x0 = oracle.start_vector(A.n_cols, 1)
    ro = oracle.projected_adam(A, pa.SIGMA_MAX, 200, x_init=x0, **HYPER)
    with pa.create(A, grid_blocks=12, **SINGLE) as h:
        runs = [h.run(pa.SIGMA_MAX, 200, x0, **HYPER)["x_last"] for _ in range(6)]
    for k, x in enumerate(runs[1:], 1):
        assert np.array_equal(x, runs[0]), f"run {k} differs from run 0"
    assert np.linalg.norm(runs[0] - ro.x_last) < 1e-12


def test_estimate_matches_three_phase_kernel():
    """A full estimate: sigma_max agrees with the three-phase kernel's and the
    oracle's to 1e-10 (both converge), and each x_min scores its sigma."""
    A = synth.hydro_operator(21, seed=1)
    with pa.create(A, grid_blocks=6, **SINGLE) as h:
        r = h.estimate(pa.SIGMA_MAX, 1500, seed=1, **HYPER)
        xg = h.get_vector(pa.SIGMA_MAX)
    with pa.create(A, engine=pa.ENGINE_GRID) as h:
        r3 = h.estimate(pa.SIGMA_MAX, 1500, seed=1, **HYPER)
    ro = oracle.estimate(A, 1500, 1, seed=1, **HYPER)
    assert abs(r["sigma_max"] / ro["sigma_max"] - 1) <= 1e-10
    assert abs(r["sigma_max"] / r3["sigma_max"] - 1) <= 1e-10
    assert abs(oracle.sigma(A, xg) / r["sigma_max"] - 1) <= 1e-12


def test_unsupported_inputs_are_refused():
    # rectangular: no shared row/position ownership
    with pa.create(CASES["rect_tall"](), **SINGLE) as h:
        with pytest.raises(pa.PAError) as ei:
            h.estimate(pa.SIGMA_MAX, 10)
        assert ei.value.status == -9
        with pytest.raises(pa.PAError) as ei:
            h.spmv_ata(np.ones(h.n_cols))
        assert ei.value.status == -9
    # FP64 only
    with pa.create(CASES["hydro21"](), precision=pa.MIXED, **SINGLE) as h:
        with pytest.raises(pa.PAError) as ei:
            h.estimate(pa.SIGMA_MAX, 10)
        assert ei.value.status == -9
    # a row longer than 255 entries
    n = 300
    rows = np.concatenate([np.zeros(n, np.int64), np.arange(1, n)])
    cols = np.concatenate([np.arange(n), np.arange(1, n)])
    A = synth.from_coo(rows, cols, np.ones(rows.size), n, n)
    with pa.create(A, **SINGLE) as h:
        with pytest.raises(pa.PAError) as ei:
            h.estimate(pa.SIGMA_MAX, 10)
        assert ei.value.status == -9


def test_edge_cases():
    # 1 x 1
    with pa.create(synth.diag_csr([-4.0]), **SINGLE) as h:
        r = h.estimate(pa.BOTH, 5, seed=1)
        assert r["sigma_max"] == 4.0 and r["sigma_min"] == 4.0 and r["kappa"] == 1.0
    # empty rows and columns, more CTAs than non-empty rows
    M = np.zeros((200, 200))
    M[0, 1], M[2, 3], M[4, 4], M[150, 7], M[7, 150] = 2.0, -1.0, 3.0, 0.5, -0.25
    A = synth.from_coo(*np.nonzero(M), M[np.nonzero(M)], 200, 200)
    x0 = oracle.start_vector(200, 2)
    ro = oracle.projected_adam(A, oracle.SIGMA_MAX, 30, x_init=x0, **HYPER)
    with pa.create(A, grid_blocks=7, **SINGLE) as h:
        rg = h.run(pa.SIGMA_MAX, 30, x0, **HYPER)
        z = h.spmv_ata(x0)
    assert np.linalg.norm(rg["x_last"] - ro.x_last) <= 1e-12
    assert np.allclose(z, M.T @ (M @ x0), rtol=1e-15, atol=1e-15)


# --------------------------------------------------- full size (C2) ---

@pytest.fixture(scope="module")
def hydro401():
    return synth.hydro_operator(401, n_incl=8, eta_lo=1e18, eta_hi=1e24, seed=2)


def test_full_size_ata_product(hydro401):
    """Every entry of A^T (A x) on the 964,806-row operator, in the grid the
    engine runs."""
    A = hydro401
    x = oracle.start_vector(A.n_cols, 5)
    with pa.create(A, **SINGLE) as h:
        z = h.spmv_ata(x)
        info = h.single_pass_info()
    y = oracle.spmv(A, x)
    assert np.all(np.abs(z - oracle.spmv_t(A, y)) <= _ata_bound(A, x, y))
    assert info["plan_entries"] == A.nnz


@pytest.mark.parametrize("mode", [pa.SIGMA_MAX, pa.SIGMA_MIN])
def test_full_size_first_iterates(hydro401, mode):
    A = hydro401
    T = 40
    x0 = oracle.start_vector(A.n_cols, 1)
    ro = oracle.projected_adam(A, mode, T, x_init=x0, trace_L=True, **HYPER)
    with pa.create(A, **SINGLE) as h:
        rg = h.run(mode, T, x0, trace_L=True, **HYPER)
    assert np.linalg.norm(rg["x_last"] - ro.x_last) <= 1e-10
    Lo = ro.L_trace
    assert np.max(np.abs(rg["L_trace"] - Lo) / np.maximum(1, np.abs(Lo))) <= 1e-10
