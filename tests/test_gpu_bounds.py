"""pa_error_bounds (the paper's Theorems 1-4) against the oracle.

The residual entries are computed by the same Dot2 algorithm in the same
order on both sides (its error-free transformations are exact with or
without FMA), so only the order of the three norm sums differs: norms and
bounds must agree to 1e-13 relative; the singularity flag exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2409_11515_gb300 import build, pa, synth

pytestmark = pytest.mark.gpu
HYPER = dict(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12)
KEYS = pa.ERROR_BOUND_KEYS


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    pa.load()


def _system(A, seed, noise):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(A.n_cols)
    b = oracle.spmv(A, x)
    x_hat = x * (1 + noise * rng.standard_normal(A.n_cols))
    return x_hat, b


def _close(g, o, rel=1e-13):
    for k in KEYS:
        if np.isinf(o[k]) or o[k] == 0.0:
            assert g[k] == o[k], k
        else:
            assert abs(g[k] / o[k] - 1) <= rel, (k, g[k], o[k])


@pytest.mark.parametrize("make", [lambda: synth.hydro_operator(21, seed=1),
                                  lambda: synth.random_sparse(3000, 9, seed=3, diag_boost=4.0),
                                  lambda: synth.random_sparse(700, 5, seed=4, n_cols=500)],
                         ids=["hydro21", "random", "rect"])
@pytest.mark.parametrize("noise", [0.0, 1e-12, 1e-3])
def test_error_bounds_match_oracle(make, noise):
    A = make()
    x_hat, b = _system(A, 5, noise)
    kappa, norm_a = 3.7e8, 2.5e3
    o = oracle.error_bounds(A, x_hat, b, kappa, norm_a)
    with pa.create(A) as h:
        g = h.error_bounds(x_hat, b, kappa, norm_a)
    _close(g, o)


def test_compensated_residual_on_cancelling_row():
    A = synth.from_coo([0, 0, 0, 1], [0, 1, 2, 1], [1e16, 1.0, -1e16, 2.0], 2, 3)
    with pa.create(A) as h:
        g = h.error_bounds(np.ones(3), np.array([0.0, 2.0]), kappa=1.0, norm_a=1.0)
    assert g["residual_norm"] == 1.0


def test_defaults_from_the_handle_and_device_pointers():
    torch = pytest.importorskip("torch")
    A = synth.hydro_operator(13, seed=1)
    x_hat, b = _system(A, 9, 1e-8)
    with pa.create(A) as h:
        with pytest.raises(pa.PAError):
            h.error_bounds(x_hat, b)  # no estimates yet
        r = h.estimate(pa.BOTH, 300, seed=1, **HYPER)
        g = h.error_bounds(x_hat, b)
        e = h.error_bounds(x_hat, b, r["kappa"], r["sigma_max"])
        dev = torch.device("cuda:0")
        d = h.error_bounds(torch.from_numpy(x_hat).to(dev), torch.from_numpy(b).to(dev),
                           r["kappa"], r["sigma_max"])
    assert g == e == d
    _close(g, oracle.error_bounds(A, x_hat, b, r["kappa"], r["sigma_max"]))


def test_numerical_singularity_flag():
    A = synth.laplacian_1d(50)
    x_hat, b = _system(A, 2, 0.0)
    with pa.create(A) as h:
        assert h.error_bounds(x_hat, b, 1e15, 4.0)["singular"] == 0.0
        assert h.error_bounds(x_hat, b, 2.0 ** 53, 4.0)["singular"] == 1.0
        assert h.error_bounds(x_hat, b, 1e8, 4.0, u=2.0 ** -24)["singular"] == 1.0


def test_full_size_error_bounds():
    A = synth.hydro_operator(401, n_incl=8, eta_lo=1e18, eta_hi=1e24, seed=2)
    x_hat, b = _system(A, 1, 1e-10)
    o = oracle.error_bounds(A, x_hat, b, 1e20, 1e19)
    with pa.create(A) as h:
        g = h.error_bounds(x_hat, b, 1e20, 1e19)
    _close(g, o, rel=1e-12)
