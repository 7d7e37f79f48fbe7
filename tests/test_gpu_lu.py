"""sigma_min through ||A^{-1}|| with given LU factors (the paper's Algorithm 2
inside Algorithm 1) on the GPU, against the oracle.

The GPU sums each row of a triangular solve with a warp butterfly and FMA,
another rounding order than the oracle's plain substitution; the route is
insensitive to that (builds of the oracle with FMA contraction or with rows
summed backwards agree with it to 1e-15 over 100 iterations).  Bars: iterates
and L_t within 1e-10 for 100 iterations, the tracked iteration equal, sigma
within 1e-12; the converged sigma_min within 1e-10 of 1 / sigma_max of the
dense LU inverse.
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


def lu_factors(A, spec="COLAMD"):
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


CASES = {
    "hydro13": lambda: synth.hydro_operator(13, seed=1),
    "hydro21": lambda: synth.hydro_operator(21, seed=1),
    "random": lambda: synth.random_sparse(1500, 7, seed=3, diag_boost=3.0),
    "lap2d_12": lambda: synth.laplacian_2d(12),
}


# engine AUTO runs these small factors on one CTA (level steps, kernel 4);
# engine GRID forces the grid kernel with per-row waits (kernel 5), CLUSTER
# the cluster kernel with the solve vectors in distributed shared memory (7)
@pytest.mark.parametrize("engine,kernel", [(pa.ENGINE_AUTO, 4), (pa.ENGINE_GRID, 5),
                                           (pa.ENGINE_CLUSTER, 7)],
                         ids=["one_cta", "grid", "cluster"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_lu_route_iterates_match_oracle(name, engine, kernel):
    A = CASES[name]()
    Lf, Uf, p, q = lu_factors(A)
    T = 100
    x0 = oracle.start_vector(A.n_cols, 7)
    ro = oracle.projected_adam_lu(Lf, Uf, p, q, T, x0, n_trace=T, trace_L=True, **HYPER)
    with pa.create(A, engine=engine) as h:
        h.attach_lu(Lf, Uf, p, q)
        ri = h.lu_route_info()
        rg = h.run(pa.SIGMA_MIN_LU, T, x0, trace_L=True, n_trace=T, **HYPER)
        xv = h.get_vector(pa.SIGMA_MIN_LU)
        assert h.last_run_info()["kernel"] == kernel
    assert ri["route"] == {4: 0, 5: 1, 7: 2}[kernel]
    if kernel == 7:  # small factors: 16 CTAs keeping the final values
        assert ri["ctas"] == 16 and ri["fin"] == 1 and ri["cap"] >= 160
    assert rg["status"] == ro.status == 0
    err_x = np.linalg.norm(rg["x_trace"] - ro.x_trace, axis=1)
    err_L = np.abs(rg["L_trace"] - ro.L_trace) / np.maximum(1.0, np.abs(ro.L_trace))
    assert np.max(err_x) <= 1e-10, np.max(err_x)
    assert np.max(err_L) <= 1e-10
    assert rg["t_min"] == ro.t_min
    assert abs(rg["sigma"] / ro.sigma_min - 1) <= 1e-12
    assert np.array_equal(xv, rg["x_min"])
    assert np.linalg.norm(rg["x_min"] - ro.x_min) <= 1e-10


@pytest.mark.parametrize("engine", [pa.ENGINE_AUTO, pa.ENGINE_GRID, pa.ENGINE_CLUSTER],
                         ids=["auto", "grid", "cluster"])
@pytest.mark.parametrize("name", ["hydro13", "hydro21"])
def test_lu_route_kappa_matches_dense_inverse(name, engine):
    """kappa ~ 1e22: Algorithm 2's sigma_min against 1 / sigma_max of the
    dense LU inverse; sigma_max of Algorithm 1 against the dense SVD."""
    A = CASES[name]()
    Lf, Uf, p, q = lu_factors(A)
    D = synth.csr_to_dense(A)
    smin_ref = 1.0 / np.linalg.svd(np.linalg.inv(D), compute_uv=False)[0]
    smax_ref = np.linalg.svd(D, compute_uv=False)[0]
    with pa.create(A, engine=engine) as h:
        h.attach_lu(Lf, Uf, p, q)
        r = h.estimate(pa.BOTH_LU, 1000, seed=1, **HYPER)
    assert r["status"] == 0
    assert abs(r["sigma_min"] / smin_ref - 1) <= 1e-10, (r["sigma_min"], smin_ref)
    assert abs(r["sigma_max"] / smax_ref - 1) <= 1e-6
    assert r["kappa"] == pytest.approx(r["sigma_max"] / r["sigma_min"], rel=1e-15)
    assert r["kappa"] > 1e20


def test_identity_permutations_and_diagonal_factors():
    d = np.array([3.0, -0.5, 7.0, 0.25, 2.0, -4.0])
    A = synth.diag_csr(d)
    I = synth.diag_csr(np.ones(6))
    with pa.create(A) as h:
        h.attach_lu(I, A)  # L = I, U = diag(d), P = Q = identity
        r = h.estimate(pa.SIGMA_MIN_LU, 300, seed=2, **HYPER)
    assert r["sigma_min"] == pytest.approx(0.25, rel=1e-14)


def test_device_factors_equal_host_factors():
    torch = pytest.importorskip("torch")
    A = CASES["hydro13"]()
    Lf, Uf, p, q = lu_factors(A)
    dev = torch.device("cuda:0")

    def tens(T):
        return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                     for a in (T.row_ptr, T.col, T.val)) + (T.n_rows, T.n_cols)

    with pa.create(A) as h:
        h.attach_lu(Lf, Uf, p, q)
        r1 = h.estimate(pa.SIGMA_MIN_LU, 200, seed=3, **HYPER)
        h.attach_lu(tens(Lf), tens(Uf), torch.from_numpy(p).to(dev), torch.from_numpy(q).to(dev))
        r2 = h.estimate(pa.SIGMA_MIN_LU, 200, seed=3, **HYPER)
    assert r1["sigma_min"] == r2["sigma_min"]


def test_attach_errors():
    A = CASES["hydro13"]()
    Lf, Uf, p, q = lu_factors(A)
    with pa.create(A) as h:
        with pytest.raises(pa.PAError):
            h.estimate(pa.SIGMA_MIN_LU, 10, seed=1, **HYPER)  # nothing attached
        with pytest.raises(pa.PAError):
            h.attach_lu(Uf, Lf, p, q)  # swapped: not lower / upper triangular
        bad = p.copy()
        bad[0] = bad[1]
        with pytest.raises(pa.PAError):
            h.attach_lu(Lf, Uf, bad, q)  # not a permutation
        Z = synth.CSR(Uf.row_ptr, Uf.col, Uf.val.copy(), Uf.n_rows, Uf.n_cols)
        first_diag = Z.row_ptr[0] + int(np.nonzero(Z.col[Z.row_ptr[0]:Z.row_ptr[1]] == 0)[0][0])
        Z.val[first_diag] = 0.0
        with pytest.raises(pa.PAError):
            h.attach_lu(Lf, Z, p, q)  # zero pivot
        h.attach_lu(Lf, Uf, p, q)  # still usable after the refusals
        assert h.estimate(pa.SIGMA_MIN_LU, 10, seed=1, **HYPER)["status"] == 0
    with pa.create(synth.random_sparse(30, 4, seed=1, n_cols=20)) as h:
        with pytest.raises(pa.PAError):
            h.attach_lu(Lf, Uf)  # not square


def test_batched_lu_route_equals_single_handle_runs():
    """pa_estimate_batched with PA_BOTH_LU: sigma_min of item (i, r) through
    the LU route in its own CTA equals the single-handle estimate from the
    same seed bit for bit; sigma_max equals the SpMM path's."""
    mats = [synth.hydro_operator(nx, seed=nx) for nx in (7, 9, 13)]
    k, seed, it = 3, 5, (300, 600)
    hs = [pa.create(A) for A in mats]
    try:
        for h, A in zip(hs, mats):
            h.attach_lu(*lu_factors(A))
        rb = pa.estimate_batched(hs, pa.BOTH_LU, k, it, seed=seed, **HYPER)
        rm = pa.estimate_batched(hs, pa.SIGMA_MAX, k, it, seed=seed, **HYPER)
        assert rb["status"] == 0 and np.all(rb["item_status"] == 0)
        assert np.array_equal(rb["sigma_max"], rm["sigma_max"])
        for i, (h, A) in enumerate(zip(hs, mats)):
            smin_ref = 1.0 / np.linalg.svd(np.linalg.inv(synth.csr_to_dense(A)),
                                           compute_uv=False)[0]
            for r in range(k):
                s_ir = oracle.splitmix64_at(seed, i * k + r)
                single = h.estimate(pa.SIGMA_MIN_LU, it[1], seed=s_ir, **HYPER)
                assert rb["sigma_min"][i, r] == single["sigma_min"]
                assert abs(rb["sigma_min"][i, r] / smin_ref - 1) <= 1e-8  # 600 iterations
                assert rb["kappa"][i, r] == rb["sigma_max"][i, r] / rb["sigma_min"][i, r]
        only = pa.estimate_batched(hs, pa.SIGMA_MIN_LU, k, it, seed=seed, **HYPER)
        assert np.array_equal(only["sigma_min"], rb["sigma_min"])
        assert np.all(np.isnan(only["sigma_max"]))
    finally:
        for h in hs:
            h.destroy()


def test_batched_lu_needs_factors_on_every_handle():
    mats = [synth.hydro_operator(7, seed=1), synth.hydro_operator(9, seed=2)]
    hs = [pa.create(A) for A in mats]
    try:
        hs[0].attach_lu(*lu_factors(mats[0]))
        with pytest.raises(pa.PAError):
            pa.estimate_batched(hs, pa.BOTH_LU, 2, (10, 10), seed=1, **HYPER)
    finally:
        for h in hs:
            h.destroy()


@pytest.fixture(scope="module")
def hydro129_lu():
    A = synth.hydro_operator(129, seed=7)
    Lf, Uf, p, q = lu_factors(A)
    T = 10
    x0 = oracle.start_vector(A.n_cols, 1)
    ro = oracle.projected_adam_lu(Lf, Uf, p, q, T, x0, n_trace=T, trace_L=True, **HYPER)
    return A, (Lf, Uf, p, q), x0, ro


# AUTO: past one CTA's shared memory the cluster kernel (7) takes these
# factors; GRID forces the grid kernel (5)
@pytest.mark.parametrize("engine,kernel", [(pa.ENGINE_AUTO, 7), (pa.ENGINE_GRID, 5)],
                         ids=["cluster", "grid"])
def test_lu_route_100k_rows_matches_oracle(hydro129_lu, engine, kernel):
    """The 129 x 129 operator (99,846 rows; COLAMD factors with about 27M
    non-zeros and 5,400 levels per system): the solve vector no longer fits
    in one CTA's shared memory.  Iterates and L_t for t <= 10 and sigma after
    10 iterations against the oracle; the run is reproducible."""
    A, (Lf, Uf, p, q), x0, ro = hydro129_lu
    T = 10
    with pa.create(A, engine=engine) as h:
        h.attach_lu(Lf, Uf, p, q)
        rg = h.run(pa.SIGMA_MIN_LU, T, x0, trace_L=True, n_trace=T, **HYPER)
        assert h.last_run_info()["kernel"] == kernel
        rg2 = h.run(pa.SIGMA_MIN_LU, T, x0, **HYPER)
    assert rg["status"] == ro.status == 0
    err_x = np.linalg.norm(rg["x_trace"] - ro.x_trace, axis=1)
    err_L = np.abs(rg["L_trace"] - ro.L_trace) / np.maximum(1.0, np.abs(ro.L_trace))
    assert np.max(err_x) <= 1e-10, np.max(err_x)
    assert np.max(err_L) <= 1e-10
    assert rg["t_min"] == ro.t_min
    assert abs(rg["sigma"] / ro.sigma_min - 1) <= 1e-12
    assert np.array_equal(rg2["x_last"], rg["x_last"])


def _lu_parity(A, engine, T, route, fin):
    """The LU route's iterates, L_t and sigma after T iterations against the
    oracle on A's COLAMD factors, with the route pa_lu_route_info reports."""
    Lf, Uf, p, q = lu_factors(A)
    x0 = oracle.start_vector(A.n_cols, 1)
    ro = oracle.projected_adam_lu(Lf, Uf, p, q, T, x0, n_trace=T, trace_L=True, **HYPER)
    with pa.create(A, engine=engine) as h:
        h.attach_lu(Lf, Uf, p, q)
        ri = h.lu_route_info()
        assert ri["route"] == route and ri["fin"] == fin, ri
        rg = h.run(pa.SIGMA_MIN_LU, T, x0, trace_L=True, n_trace=T, **HYPER)
        assert h.last_run_info()["kernel"] == {0: 4, 1: 5, 2: 7}[route]
    assert rg["status"] == ro.status == 0
    err_x = np.linalg.norm(rg["x_trace"] - ro.x_trace, axis=1)
    err_L = np.abs(rg["L_trace"] - ro.L_trace) / np.maximum(1.0, np.abs(ro.L_trace))
    assert np.max(err_x) <= 1e-10, np.max(err_x)
    assert np.max(err_L) <= 1e-10
    assert rg["t_min"] == ro.t_min
    assert abs(rg["sigma"] / ro.sigma_min - 1) <= 1e-12


def test_lu_route_cluster_from_8192_rows():
    """The 41 x 41 operator (10,086 rows): the solve vector fits one CTA's
    shared memory, but from 8,192 rows on engine AUTO takes the cluster
    (faster there), with the final values kept; smaller factors (5,766 rows)
    stay on one CTA."""
    _lu_parity(synth.hydro_operator(41, seed=7), pa.ENGINE_AUTO, 20, route=2, fin=1)
    A = synth.hydro_operator(31, seed=7)  # 5,766 rows
    with pa.create(A) as h:
        h.attach_lu(*lu_factors(A))
        assert h.lu_route_info() == dict(route=0, ctas=0, cap=0, fin=0)


def test_lu_route_214k_rows_release_barrier():
    """The 189 x 189 operator (214,326 rows; COLAMD factors with about 72M
    non-zeros): the final-value arrays no longer fit next to the solve vector
    in the cluster's shared memory, so the cluster's steps end with a release
    barrier instead.  Iterates, L_t and sigma after 5 iterations against the
    oracle."""
    _lu_parity(synth.hydro_operator(189, seed=7), pa.ENGINE_AUTO, 5, route=2, fin=0)
