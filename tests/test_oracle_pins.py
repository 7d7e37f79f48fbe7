"""Pins of the CPU oracle against facts outside itself (no GPU).

Each test pins one part of the oracle (the paper's Eq. nabla_loss and
Algorithm 1) to something the paper or mathematics fixes: exact integer
products, rational arithmetic, finite differences, closed-form singular
values, dense SVD, the explicit-sum form of Adam's moment recursions and
invariances of the loss.  ``test_mutants_are_caught`` plants mistakes in a
copy of the oracle source and checks that these pins catch each one.
"""
import json
import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2409_11515_gb300 import synth

GOLDEN = Path(__file__).resolve().parent / "golden"
CF = json.loads((GOLDEN / "closed_forms.json").read_text())
B1, B2, LR, EPS = 0.9, 0.999, 1e-2, 1e-12


def _int_matrix(m, n, seed, density=0.4):
    rng = np.random.default_rng(seed)
    M = rng.integers(-9, 10, size=(m, n)).astype(np.float64)
    M[rng.random((m, n)) > density] = 0.0
    return M


# ----------------------------------------------------------------- RNG ---

def test_splitmix64_known_answers():
    for line in (GOLDEN / "splitmix64_seed0.txt").read_text().splitlines():
        if not line or line.startswith("#"):
            continue
        i, hx = line.split()
        assert oracle.splitmix64_at(0, int(i)) == int(hx, 16)


def test_start_vector_unit_and_uniform():
    x = oracle.start_vector(100000, 42)
    assert abs(np.linalg.norm(x) - 1.0) < 1e-14
    # raw entries 2u-1 are uniform on [-1, 1): check mean / second moment
    raw = x * np.sqrt(100000 / 3.0) * (1.0 / np.sqrt(np.mean((x * np.sqrt(100000 / 3.0)) ** 2)))
    assert abs(np.mean(raw)) < 0.02
    assert not np.array_equal(oracle.start_vector(1000, 1), oracle.start_vector(1000, 2))


# ------------------------------------------------------------ products ---

@pytest.mark.parametrize("shape", [(7, 7), (13, 5), (5, 13), (40, 40)])
def test_spmv_exact_on_integers(shape):
    M = _int_matrix(*shape, seed=sum(shape))
    A = synth.from_coo(*np.nonzero(M), M[np.nonzero(M)], *shape)
    x = np.random.default_rng(1).integers(-50, 50, shape[1]).astype(np.float64)
    y = np.random.default_rng(2).integers(-50, 50, shape[0]).astype(np.float64)
    assert np.array_equal(oracle.spmv(A, x), M @ x)
    assert np.array_equal(oracle.spmv_t(A, y), M.T @ y)


def test_spmv_empty_rows_and_columns():
    M = np.zeros((6, 6))
    M[1, 2] = 3.0
    M[4, 0] = -2.0
    A = synth.from_coo(*np.nonzero(M), M[np.nonzero(M)], 6, 6)
    x = np.arange(1.0, 7.0)
    assert np.array_equal(oracle.spmv(A, x), M @ x)
    assert np.array_equal(oracle.spmv_t(A, x), M.T @ x)


def test_dd_products_match_rational_arithmetic():
    # rows built to cancel: terms of size 1e16 summing to O(1)
    rng = np.random.default_rng(5)
    n = 12
    x = rng.uniform(0.5, 1.5, n)
    rows, cols, vals = [], [], []
    for i in range(n):
        big = rng.uniform(1, 2) * 1e16
        c = [(i + k) % n for k in range(4)]
        rows += [i, i, i, i]
        cols += c
        # the first two products cancel to within their own rounding error
        vals += [big, -big * x[c[0]] / x[c[1]], rng.uniform(-1, 1), rng.uniform(-1, 1) * 1e-8]
    A = synth.from_coo(rows, cols, vals, n, n)
    hi, lo = oracle.spmv(A, x, dd=True)
    plain = oracle.spmv(A, x)
    for i in range(n):
        exact = sum(Fraction(A.val[k]) * Fraction(x[A.col[k]])
                    for k in range(A.row_ptr[i], A.row_ptr[i + 1]))
        ref = float(exact)
        # Dot2: |hi - exact| <= u|exact| + gamma^2 * sum|terms|  (tiny here)
        terms = sum(abs(A.val[k] * x[A.col[k]]) for k in range(A.row_ptr[i], A.row_ptr[i + 1]))
        assert abs(hi[i] - ref) <= 2.3e-16 * abs(ref) + 1e-30 * terms + 1e-300
        assert abs(Fraction(hi[i]) + Fraction(lo[i]) - exact) <= Fraction(1e-28) * Fraction(terms)
    # plain FP64 loses most digits on these rows, so the test does separate them
    assert np.max(np.abs(plain - hi) / np.abs(hi)) > 1e-6
    # transposed dd product against rational arithmetic
    z = oracle.spmv_t(A, hi, lo)
    for j in range(n):
        exact = Fraction(0)
        for i in range(n):
            for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
                if A.col[k] == j:
                    exact += Fraction(A.val[k]) * (Fraction(hi[i]) + Fraction(lo[i]))
        assert abs(z[j] - float(exact)) <= 4.5e-16 * abs(float(exact)) + 1e-300


# ------------------------------------------------------------ gradient ---

@pytest.mark.parametrize("mode", [oracle.SIGMA_MAX, oracle.SIGMA_MIN])
@pytest.mark.parametrize("loss", [oracle.LOSS_LOGRATIO, oracle.LOSS_QUADRATIC])
def test_gradient_matches_finite_differences(mode, loss):
    rng = np.random.default_rng(3)
    M = rng.standard_normal((9, 7))
    A = synth.dense_csr(M)
    x = rng.standard_normal(7)

    def L(v):  # the loss as defined in the paper (and its negation / the quadratic reading)
        if loss == oracle.LOSS_LOGRATIO:
            val = math.log(np.linalg.norm(v)) - math.log(np.linalg.norm(M @ v))
            return val if mode == oracle.SIGMA_MAX else -val
        q = float(np.dot(M @ v, M @ v))
        return -q if mode == oracle.SIGMA_MAX else q

    Lo, g = oracle.loss_grad(A, x, mode, loss)
    assert abs(Lo - L(x)) <= 1e-13 * max(1.0, abs(L(x)))
    h = 1e-6
    fd = np.array([(L(x + h * e) - L(x - h * e)) / (2 * h) for e in np.eye(7)])
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-8 * np.max(np.abs(fd)))


def test_logratio_gradient_is_tangent():
    # L is scale invariant, so x . grad L(x) = 0 (Euler's theorem, degree 0)
    rng = np.random.default_rng(8)
    A = synth.random_sparse(50, 5, seed=8, diag_boost=3.0)
    x = rng.standard_normal(50)
    _, g = oracle.loss_grad(A, x, oracle.SIGMA_MAX)
    assert abs(np.dot(x, g)) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(g)


# ------------------------------------------------ Adam steps, explicitly ---

def _fd_grad(M, v, mode):
    def L(u):
        val = math.log(np.linalg.norm(u)) - math.log(np.linalg.norm(M @ u))
        return val if mode == oracle.SIGMA_MAX else -val
    h = 1e-6
    return np.array([(L(v + h * e) - L(v - h * e)) / (2 * h) for e in np.eye(v.size)])


@pytest.mark.parametrize("mode", [oracle.SIGMA_MAX, oracle.SIGMA_MIN])
def test_first_five_steps_match_explicit_adam(mode):
    """x_t from the closed (explicit-sum) form of Adam's moments with
    finite-difference gradients: m_t = (1-b1) sum_k b1^(t-k) g_k, likewise v_t
    with g_k^2, bias-corrected by 1 - b^t; then the tangent projection and the
    normalisation of Algorithm 1."""
    rng = np.random.default_rng(21)
    M = rng.standard_normal((8, 8)) + 2 * np.eye(8)
    A = synth.dense_csr(M)
    x0 = oracle.start_vector(8, 9)
    T = 5
    r = oracle.projected_adam(A, mode, T, LR, B1, B2, EPS, x_init=x0, n_trace=T)
    xs = [x0] + [r.x_trace[t] for t in range(T)]
    gs = []
    for t in range(1, T + 1):
        x = xs[t - 1]
        gs.append(_fd_grad(M, x, mode))
        assert np.min(np.abs(gs[-1])) > 1e-5  # well away from FD noise and eps
        w1 = np.array([B1 ** (t - k) for k in range(1, t + 1)])
        w2 = np.array([B2 ** (t - k) for k in range(1, t + 1)])
        G = np.array(gs)
        mh = (1 - B1) * (w1 @ G) / (1 - B1 ** t)
        vh = (1 - B2) * (w2 @ (G * G)) / (1 - B2 ** t)
        dx = LR * mh / (np.sqrt(vh) + EPS)
        dx = dx - np.dot(x, dx) * x
        xn = x - dx
        xn = xn / np.linalg.norm(xn)
        assert np.max(np.abs(xn - xs[t])) < 1e-8, t
    # t = 1 is projected sign descent: |dx_i| = LR for every coordinate
    d1 = LR * np.sign(gs[0])
    x1 = x0 - (d1 - np.dot(x0, d1) * x0)
    assert np.max(np.abs(x1 / np.linalg.norm(x1) - xs[1])) < 1e-10


# ------------------------------------------------------- closed forms ---

@pytest.mark.parametrize("case", CF["lap1d"], ids=lambda c: f"n{c['n']}")
def test_laplacian_1d_kappa(case):
    A = synth.laplacian_1d(case["n"])
    r = oracle.estimate(A, 3000, 3000, seed=1)
    assert r["status_max"] == 0 and r["status_min"] == 0
    assert abs(r["sigma_max"] / case["sigma_max"] - 1) < 1e-6
    assert abs(r["sigma_min"] / case["sigma_min"] - 1) < 1e-6
    assert abs(r["kappa"] / case["kappa"] - 1) < 1e-6


@pytest.mark.parametrize("case", CF["lap2d"], ids=lambda c: f"N{c['N']}")
def test_laplacian_2d_kappa(case):
    A = synth.laplacian_2d(case["N"])
    r = oracle.estimate(A, 3000, 3000, seed=3)
    assert abs(r["kappa"] / case["kappa"] - 1) < 1e-6
    assert abs(r["sigma_max"] / case["sigma_max"] - 1) < 1e-6


@pytest.mark.parametrize("case", CF["two_by_two"], ids=["a", "b"])
def test_two_by_two(case):
    A = synth.dense_csr(np.array(case["M"]))
    r = oracle.estimate(A, 2000, 2000, seed=4)
    assert abs(r["sigma_max"] / case["sigma_max"] - 1) < 1e-9
    assert abs(r["sigma_min"] / case["sigma_min"] - 1) < 1e-9


def test_diagonal_exact():
    rng = np.random.default_rng(0)
    d = rng.uniform(0.5, 2.0, 50) * np.where(rng.random(50) < 0.5, -1, 1)
    r = oracle.estimate(synth.diag_csr(d), 5000, 5000, seed=5)
    assert abs(r["sigma_max"] / np.max(np.abs(d)) - 1) < 1e-9
    assert abs(r["sigma_min"] / np.min(np.abs(d)) - 1) < 1e-9


def test_scalar_identity_never_moves():
    # A = c I: the log-ratio gradient vanishes up to round-off (|g| ~ 1e-16,
    # far below eps = 1e-12), so each step moves x by at most ~lr*|g|/eps and
    # every iterate scores sigma = |c|
    A = synth.diag_csr(np.full(30, -3.0))
    x0 = oracle.start_vector(30, 2)
    _, g = oracle.loss_grad(A, x0, oracle.SIGMA_MAX)
    assert np.max(np.abs(g)) < 1e-15
    r = oracle.projected_adam(A, oracle.SIGMA_MAX, 50, x_init=x0)
    assert np.max(np.abs(r.x_last - x0)) < 50 * LR * 1e-15 / EPS
    assert abs(r.sigma - 3.0) < 1e-15


def test_pow2_identity_exact_fixed_point_and_earliest_minimum():
    # A = 2 I: A^T A x = 4x and ||Ax||^2 = 4||x||^2 exactly, so the log-ratio
    # gradient is exactly 0, Adam's step is 0/(0 + eps) = 0, x never moves and
    # every iterate ties in L; the strict "<" of Algorithm 1 keeps t_min = 1.
    A = synth.diag_csr(np.full(16, 2.0))
    x0 = oracle.start_vector(16, 4)
    _, g = oracle.loss_grad(A, x0, oracle.SIGMA_MAX)
    assert np.all(g == 0.0)
    r = oracle.projected_adam(A, oracle.SIGMA_MAX, 20, x_init=x0, trace_L=True)
    assert np.array_equal(r.x_last, x0)
    assert np.all(r.L_trace == r.L_trace[0])
    assert r.t_min == 1
    assert r.sigma == 2.0


@pytest.mark.parametrize("n", [20, 60, 120])
def test_dense_svd_sigma_max(n):
    rng = np.random.default_rng(n)
    U, _, Vt = np.linalg.svd(rng.standard_normal((n, n)))
    S = np.logspace(0, 2, n)[::-1]
    M = (U * S) @ Vt
    r = oracle.projected_adam(synth.dense_csr(M), oracle.SIGMA_MAX, 2000, seed=11)
    assert abs(r.sigma / S[0] - 1) < 1e-9


def test_dense_svd_sigma_min_small():
    rng = np.random.default_rng(20)
    U, _, Vt = np.linalg.svd(rng.standard_normal((20, 20)))
    S = np.logspace(0, 1, 20)[::-1]
    M = (U * S) @ Vt
    r = oracle.projected_adam(synth.dense_csr(M), oracle.SIGMA_MIN, 5000, seed=11)
    assert abs(r.sigma / S[-1] - 1) < 1e-6


# --------------------------------------------------------- invariants ---

def test_unit_norm_and_tracking_invariants():
    A = synth.hydro_operator(9, seed=3)
    for mode in (oracle.SIGMA_MAX, oracle.SIGMA_MIN):
        r = oracle.projected_adam(A, mode, 300, seed=7, n_trace=300, trace_L=True)
        norms = np.linalg.norm(r.x_trace, axis=1)
        assert np.max(np.abs(norms - 1)) < 1e-14
        L = r.L_trace
        assert r.L_min == np.min(L)
        assert r.t_min == int(np.argmin(L)) + 1  # earliest minimum (strict "<")
        assert np.array_equal(r.x_min, r.x_trace[r.t_min - 1])


def test_objective_monotone_after_warmup_on_closed_form():
    A = synth.laplacian_1d(8)
    r = oracle.projected_adam(A, oracle.SIGMA_MAX, 1500, seed=1, trace_L=True)
    L = r.L_trace[200:]
    # L decreases to its floor; any rise after warm-up stays at round-off level
    assert np.all(np.diff(L) <= 1e-12 * np.abs(L[1:]) + 1e-15)


def test_pow2_scaling_gives_identical_iterates():
    A = synth.hydro_operator(7, seed=2)
    B = synth.CSR(A.row_ptr, A.col, A.val * 2.0 ** 37, A.n_rows, A.n_cols)
    for mode in (oracle.SIGMA_MAX, oracle.SIGMA_MIN):
        ra = oracle.projected_adam(A, mode, 200, seed=3)
        rb = oracle.projected_adam(B, mode, 200, seed=3)
        assert np.array_equal(ra.x_last, rb.x_last)
        assert rb.sigma == ra.sigma * 2.0 ** 37


def test_transpose_and_permutation_invariance():
    A = synth.laplacian_2d(4)
    D = synth.csr_to_dense(A)
    rng = np.random.default_rng(2)
    D = D + np.diag(rng.uniform(0, 1, 16)) + 0.3 * np.triu(rng.standard_normal((16, 16)), 1)
    perm = rng.permutation(16)
    s = np.linalg.svd(D, compute_uv=False)
    for M in (D, D.T, D[perm][:, perm]):
        r = oracle.projected_adam(synth.dense_csr(M), oracle.SIGMA_MAX, 3000, seed=5)
        assert abs(r.sigma / s[0] - 1) < 1e-9


def test_rayleigh_sandwich_on_hydro():
    A = synth.hydro_operator(21, seed=1)
    M = synth.csr_to_dense(A)
    smax = np.linalg.svd(M, compute_uv=False)[0]
    cn = np.linalg.norm(M, axis=0)
    rmax = oracle.projected_adam(A, oracle.SIGMA_MAX, 2000, seed=1)
    rmin = oracle.projected_adam(A, oracle.SIGMA_MIN, 2000, seed=1)
    # sigma_max converges; sigma_min is an upper bound, below every column norm
    assert abs(rmax.sigma / smax - 1) < 1e-6
    assert rmax.sigma >= np.max(cn) * (1 - 1e-15)
    assert rmax.sigma <= math.sqrt(np.max(np.abs(M).sum(0)) * np.max(np.abs(M).sum(1)))
    assert rmin.sigma <= np.max(cn)
    assert rmin.sigma > 0


def test_singular_matrix_status():
    M = np.array([[1.0, 2.0], [2.0, 4.0]])
    A = synth.dense_csr(M)
    # start exactly in the null space: sigma_min = 0 at x_init
    x0 = np.array([2.0, -1.0]) / math.sqrt(5)
    r = oracle.projected_adam(A, oracle.SIGMA_MIN, 10, x_init=x0)
    assert r.status == oracle.SINGULAR and r.sigma == 0.0 and r.t_min == 0
    Z = synth.CSR(np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0), 3, 3)
    r = oracle.projected_adam(Z, oracle.SIGMA_MAX, 10, seed=1)
    assert r.status == oracle.SINGULAR


def test_nonfinite_status():
    A = synth.diag_csr([1.0, np.nan, 2.0])
    r = oracle.projected_adam(A, oracle.SIGMA_MAX, 10, seed=1)
    assert r.status == oracle.NONFINITE


# ------------------------------------------------------ equilibration ---

def test_equilibration_pow2_exact():
    A = synth.hydro_operator(9, seed=4)
    dr, dc, vh = oracle.equilibrate_pow2(A)
    for d in (dr, dc):
        m, e = np.frexp(d)
        assert np.all(m == 0.5)
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    # exact reconstruction (powers of two)
    assert np.array_equal(vh * dr[rows] * dc[A.col], A.val)
    M = synth.csr_to_dense(A)
    rn = np.linalg.norm(M, axis=1)
    ratio = rn / dr
    assert np.all(ratio >= 2 ** -0.5 - 1e-12) and np.all(ratio <= 2 ** 0.5 + 1e-12)
    cn = np.linalg.norm(M / dr[:, None], axis=0)
    ratio = cn / dc
    assert np.all(ratio >= 2 ** -0.5 - 1e-12) and np.all(ratio <= 2 ** 0.5 + 1e-12)


def test_equilibrated_hydro_sigma_max_matches_dense_svd():
    """The paper's scaled system A_hat = D_r^-1 A D_c^-1 (kappa ~ 2.5e4 here,
    against ~1e20 unscaled): Algorithm 1's sigma_max agrees with the dense SVD.
    sigma_min of the direct route only bounds the truth from above (Rayleigh)."""
    A = synth.hydro_operator(13, seed=1)
    dr, dc, vh = oracle.equilibrate_pow2(A)
    S = synth.CSR(A.row_ptr, A.col, vh, A.n_rows, A.n_cols)
    sv = np.linalg.svd(synth.csr_to_dense(S), compute_uv=False)
    x0 = oracle.start_vector(A.n_cols, 1)
    r = oracle.projected_adam(S, oracle.SIGMA_MAX, 2000, x_init=x0, lr=LR, beta1=B1,
                              beta2=B2, eps=EPS)
    assert abs(r.sigma / sv[0] - 1) <= 1e-8
    rm = oracle.projected_adam(S, oracle.SIGMA_MIN, 500, x_init=x0, lr=LR, beta1=B1,
                               beta2=B2, eps=EPS)
    assert sv[-1] * (1 - 1e-12) <= rm.sigma <= sv[0]


# ------------------------------------ error bounds (Theorems 1-4) ---

def test_error_bounds_exact_residual_on_integers():
    """Integer A and x: b = A x is exact, so moving two entries of b by
    2^-20 gives ||r|| = 2^-20 sqrt(2) exactly."""
    M = _int_matrix(30, 30, seed=21) + 40.0 * np.eye(30)
    A = synth.dense_csr(M)
    x = np.random.default_rng(3).integers(-5, 6, size=30).astype(np.float64)
    b = M @ x
    assert np.array_equal(b, oracle.spmv(A, x))
    b[[4, 17]] += 2.0 ** -20
    e = oracle.error_bounds(A, x, b, kappa=2.0, norm_a=50.0)
    assert e["residual_norm"] == np.sqrt(2.0) * 2.0 ** -20
    assert e["b_norm"] == pytest.approx(np.linalg.norm(b), rel=1e-15)
    assert e["x_hat_norm"] == pytest.approx(np.linalg.norm(x), rel=1e-15)


def test_error_bounds_residual_survives_cancellation():
    """Row (1e16, 1, -1e16) . (1, 1, 1) - 0 = 1: plain FP64 accumulation
    returns 0, the compensated residual returns the exact 1."""
    A = synth.from_coo([0, 0, 0], [0, 1, 2], [1e16, 1.0, -1e16], 1, 3)
    x = np.ones(3)
    assert oracle.spmv(A, x)[0] == 0.0
    e = oracle.error_bounds(A, x, np.zeros(1), kappa=1.0, norm_a=1.0)
    assert e["residual_norm"] == 1.0


@pytest.mark.parametrize("kappa_true", [1e2, 1e5])
def test_error_bounds_enclose_the_true_error(kappa_true):
    """Dense systems with a prescribed kappa: the true error of a perturbed
    solution lies inside every bound of Theorems 1-3 (brute force)."""
    rng = np.random.default_rng(int(kappa_true))
    n = 40
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = U @ np.diag(np.geomspace(1.0, 1.0 / kappa_true, n)) @ V.T
    A = synth.dense_csr(M)
    sv = np.linalg.svd(M, compute_uv=False)
    kappa, norm_a = sv[0] / sv[-1], sv[0]
    for trial in range(5):
        x = rng.standard_normal(n)
        b = M @ x
        x_true = np.linalg.solve(M, b)
        x_hat = x_true + 1e-6 * rng.standard_normal(n) * (10.0 ** trial)
        e = oracle.error_bounds(A, x_hat, b, kappa=kappa, norm_a=norm_a)
        err_x = np.linalg.norm(x_hat - x_true) / np.linalg.norm(x_true)
        err_xh = np.linalg.norm(x_hat - x_true) / np.linalg.norm(x_hat)
        assert e["thm1_lower"] <= err_x * (1 + 1e-9) and err_x <= e["thm1_upper"] * (1 + 1e-9)
        assert e["thm2_lower"] <= err_xh * (1 + 1e-9) and err_xh <= e["thm2_upper"] * (1 + 1e-9)
        if e["thm2_upper"] < 1:
            assert err_x <= e["thm3_upper"] * (1 + 1e-9)
        # Theorem 2's pair is tighter than Theorem 1's upper bound only up to
        # ||b|| <= ||A|| ||x||: both uppers share the factor kappa ||r||
        assert e["thm1_upper"] / e["thm1_lower"] == pytest.approx(kappa ** 2, rel=1e-12)
        assert e["thm2_upper"] / e["thm2_lower"] == pytest.approx(kappa, rel=1e-12)


def test_error_bounds_theorem4_and_singularity():
    A = synth.laplacian_1d(5)
    x = np.ones(5)
    b = oracle.spmv(A, x)
    u = 2.0 ** -53
    e = oracle.error_bounds(A, x, b, kappa=1e10, norm_a=4.0)
    assert e["thm4_rounding"] == pytest.approx(2 * u * 1e10 / (1 - 1e10 * u), rel=1e-15)
    assert e["singular"] == 0.0
    e = oracle.error_bounds(A, x, b, kappa=2.0 ** 53, norm_a=4.0)
    assert e["thm4_rounding"] == math.inf and e["singular"] == 1.0
    # single precision reading: u = 2^-24 makes kappa = 1e10 singular
    e = oracle.error_bounds(A, x, b, kappa=1e10, norm_a=4.0, u=2.0 ** -24)
    assert e["singular"] == 1.0
    # eps >= 1: Theorem 3 gives no bound
    e = oracle.error_bounds(A, x, b + 1.0, kappa=1e6, norm_a=4.0)
    assert e["thm2_upper"] >= 1 and e["thm3_upper"] == math.inf


# ------------------------------------- Algorithm 2 (sigma_min via LU) ---

def lu_factors(A, spec="COLAMD"):
    """P A Q = L U from SuperLU (scipy), as CSR factors and the permutations
    p (row i of P A is row p[i] of A) and q (column j of A Q is column q[j])."""
    sp = pytest.importorskip("scipy.sparse")
    spl = pytest.importorskip("scipy.sparse.linalg")
    n = A.n_rows
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(n, n)).tocsc()
    lu = spl.splu(S, permc_spec=spec)
    out = []
    for T in (lu.L.tocsr(), lu.U.tocsr()):
        T.sort_indices()
        out.append(synth.CSR(T.indptr.astype(np.int32), T.indices.astype(np.int32),
                             T.data.copy(), n, n))
    return out[0], out[1], np.argsort(lu.perm_r).astype(np.int32), np.argsort(lu.perm_c).astype(np.int32)


def test_triangular_solves_exact_on_integers():
    """Unit-diagonal integer triangles and integer solutions: every solve is exact."""
    rng = np.random.default_rng(8)
    n = 40
    Lm = np.tril(rng.integers(-3, 4, size=(n, n)), -1).astype(np.float64)
    Lm[rng.random((n, n)) < 0.7] = 0.0
    Lm += np.diag(rng.choice([-1.0, 1.0], size=n))
    Um = Lm.T.copy()
    x = rng.integers(-4, 5, size=n).astype(np.float64)
    Lc, Uc = synth.dense_csr(Lm), synth.dense_csr(Um)
    assert np.array_equal(oracle.triangular_solve(Lc, Lm @ x, "lower"), x)
    assert np.array_equal(oracle.triangular_solve(Uc, Um @ x, "upper"), x)
    assert np.array_equal(oracle.triangular_solve(Uc, Um.T @ x, "upper_t"), x)
    assert np.array_equal(oracle.triangular_solve(Lc, Lm.T @ x, "lower_t"), x)


def test_lu_products_match_dense_solves():
    """r = A^{-1} x and s = A^{-T} r through permuted SuperLU factors, against
    dense solves of a well-conditioned unsymmetric matrix."""
    A = synth.random_sparse(300, 7, seed=13, diag_boost=3.0)
    Lf, Uf, p, q = lu_factors(A)
    assert not np.array_equal(p, np.arange(300)) and not np.array_equal(q, np.arange(300))
    D = synth.csr_to_dense(A)
    x = np.random.default_rng(2).standard_normal(300)
    r, s = oracle.lu_products(Lf, Uf, p, q, x)
    r_ref = np.linalg.solve(D, x)
    s_ref = np.linalg.solve(D.T, r_ref)
    assert np.linalg.norm(r - r_ref) <= 1e-12 * np.linalg.norm(r_ref)
    assert np.linalg.norm(s - s_ref) <= 1e-12 * np.linalg.norm(s_ref)


def test_lu_route_iterates_equal_algorithm1_on_the_dense_inverse():
    """Algorithm 2 only changes how the products are formed: its iterates are
    Algorithm 1's (sigma_max mode) on the explicit matrix B = A^{-1}."""
    A = synth.random_sparse(120, 6, seed=17, diag_boost=3.0)
    Lf, Uf, p, q = lu_factors(A)
    B = synth.dense_csr(np.linalg.inv(synth.csr_to_dense(A)))
    x0 = oracle.start_vector(120, 4)
    T = 30
    r = oracle.projected_adam_lu(Lf, Uf, p, q, T, x0, lr=LR, beta1=B1, beta2=B2, eps=EPS,
                                 n_trace=T, trace_L=True)
    ro = oracle.projected_adam(B, oracle.SIGMA_MAX, T, x_init=x0, lr=LR, beta1=B1, beta2=B2,
                               eps=EPS, n_trace=T, trace_L=True)
    assert np.max(np.linalg.norm(r.x_trace - ro.x_trace, axis=1)) <= 1e-11
    assert np.max(np.abs(r.L_trace - ro.L_trace)) <= 1e-11
    assert r.t_min == ro.t_min
    assert abs(r.sigma / ro.sigma - 1) <= 1e-12


def test_lu_route_laplacian_closed_form():
    n = 30
    A = synth.laplacian_1d(n)
    Lf, Uf, p, q = lu_factors(A)
    r = oracle.projected_adam_lu(Lf, Uf, p, q, 500, oracle.start_vector(n, 1), lr=LR,
                                 beta1=B1, beta2=B2, eps=EPS)
    assert r.status == 0
    assert abs(r.sigma_min / (4 * np.sin(np.pi / (2 * (n + 1))) ** 2) - 1) <= 1e-12


def test_lu_route_hydro_matches_dense_inverse():
    """The hydro-mechanical operator (kappa ~ 1e22): Algorithm 2's sigma_min
    against 1 / sigma_max of the dense LU inverse, where the direct route of
    Algorithm 1 misses by orders of magnitude."""
    A = synth.hydro_operator(13, seed=1)
    Lf, Uf, p, q = lu_factors(A)
    truth = 1.0 / np.linalg.svd(np.linalg.inv(synth.csr_to_dense(A)), compute_uv=False)[0]
    x0 = oracle.start_vector(A.n_cols, 1)
    r = oracle.projected_adam_lu(Lf, Uf, p, q, 500, x0, lr=LR, beta1=B1, beta2=B2, eps=EPS,
                                 trace_L=True)
    assert r.status == 0
    assert abs(r.sigma_min / truth - 1) <= 1e-10
    # L_min tracking: the returned vector is the best scored one
    assert r.L_min == np.nanmin(r.L_trace)
    rd = oracle.projected_adam(A, oracle.SIGMA_MIN, 500, x_init=x0, lr=LR, beta1=B1, beta2=B2,
                               eps=EPS)
    assert rd.sigma > 10 * truth


# ---------------------------------------------- planted-mistake checks ---

MUTANTS = {
    "no_bias_correction": ("double mh = m[i] / bc1;", "double mh = m[i];"),
    "gradient_sign": ("gi = x[i] / q - z[i] / s;", "gi = x[i] / q + z[i] / s;"),
    "transposed_operand": ("z[col[k]] = z[col[k]] + val[k] * y[i];",
                           "z[i % n_cols] = z[i % n_cols] + val[k] * y[col[k] % n_rows];"),
    "betas_swapped": ("m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];",
                      "m[i] = beta2 * m[i] + (1.0 - beta2) * g[i];"),
    "no_projection": ("for (int64_t i = 0; i < n; ++i) dx[i] = dx[i] - c * x[i];",
                      "for (int64_t i = 0; i < n; ++i) dx[i] = dx[i] - 0.0 * c * x[i];"),
    "sqrt_dropped": ("dx[i] = lr * mh / (sqrt(vh) + eps);", "dx[i] = lr * mh / (vh + eps);"),
    "score_before_update": ("if (L < L_min) {", "if (L <= L_min) {"),
    "residual_sign": ("two_sum(s, -b[i], &t, &te);", "two_sum(s, b[i], &t, &te);"),
    "residual_uncompensated": ("    double r = s + c;\n", "    double r = s;\n"),
    "theorem2_normalised_by_b": ("out[5] = nr / (norm_a * nx);", "out[5] = nr / (norm_a * nb);"),
    "lu_permutation_inverted": ("for (int32_t i = 0; i < n; ++i) w[i] = x[f->p ? f->p[i] : i];",
                                "for (int32_t i = 0; i < n; ++i) w[f->p ? f->p[i] : i] = x[i];"),
    "lu_transpose_solve_untransposed": (
        "  po_upper_t_solve(n, f->u_rp, f->u_ci, f->u_va, u, a);",
        "  po_upper_solve(n, f->u_rp, f->u_ci, f->u_va, u, a);"),
    "lu_gradient_sign": ("g[i] = x[i] / q2 - sv[i] / rr;", "g[i] = x[i] / q2 + sv[i] / rr;"),
}


def _pins_pass():
    """A compact run of the pins above, used against a mutated oracle."""
    checks = []
    try:
        test_first_five_steps_match_explicit_adam(oracle.SIGMA_MAX)
        checks.append(True)
    except AssertionError:
        checks.append(False)
    try:
        test_gradient_matches_finite_differences(oracle.SIGMA_MAX, oracle.LOSS_LOGRATIO)
        checks.append(True)
    except AssertionError:
        checks.append(False)
    try:
        test_unit_norm_and_tracking_invariants()
        checks.append(True)
    except AssertionError:
        checks.append(False)
    try:
        test_spmv_exact_on_integers((13, 5))
        checks.append(True)
    except AssertionError:
        checks.append(False)
    try:
        test_pow2_identity_exact_fixed_point_and_earliest_minimum()
        checks.append(True)
    except AssertionError:
        checks.append(False)
    for pin in (test_lu_products_match_dense_solves, test_lu_route_laplacian_closed_form,
                test_lu_route_iterates_equal_algorithm1_on_the_dense_inverse,
                test_error_bounds_exact_residual_on_integers,
                test_error_bounds_residual_survives_cancellation,
                lambda: test_error_bounds_enclose_the_true_error(1e5)):
        try:
            pin()
            checks.append(True)
        except AssertionError:
            checks.append(False)
    return all(checks)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutants_are_caught(name, tmp_path):
    src = oracle.source_text()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, name  # a formula both loops share is mutated in both
    lib = oracle.load(oracle.compile_variant(src.replace(old, new), tmp_path / f"{name}.so"))
    with oracle.using(lib):
        assert not _pins_pass(), f"mutant {name} survived the pins"
    assert _pins_pass()  # the real oracle passes the same checks
