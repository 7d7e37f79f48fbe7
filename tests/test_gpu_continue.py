"""Checkpoint/resume through the C ABI: pa_continue resumes the handle's
latest FP64 run from its device state (x_T, Adam's moments, the iteration
count of the bias corrections, L_min and x_min).  A run of T1 iterations
continued for T2 must give the same bits as one run of T1 + T2 -- sigma,
x_min, x_last, t_min and L_min -- on the three-phase grid kernel and on the
cluster kernel, and the continued run must match the oracle's T1 + T2 run to
the iterate bar (1e-10)."""
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


@pytest.mark.parametrize("engine,kernel", [(pa.ENGINE_CLUSTER, 3), (pa.ENGINE_GRID, 0)],
                         ids=["cluster", "grid"])
@pytest.mark.parametrize("mode", [pa.SIGMA_MAX, pa.SIGMA_MIN])
def test_continue_is_bit_identical(mode, engine, kernel):
    A = synth.hydro_operator(41, seed=3)
    x0 = oracle.start_vector(A.n_cols, 2)
    T1, T2a, T2b = 70, 30, 20
    with pa.create(A, engine=engine, grid_blocks=16) as h:
        full = h.run(mode, T1 + T2a + T2b, x0, **HYPER)
        h.run(mode, T1, x0, **HYPER)
        assert h.last_run_info()["kernel"] == kernel
        h.continue_run(T2a, **HYPER)
        c = h.continue_run(T2b, **HYPER)  # a continued run can be continued
        xm = h.get_vector(mode)
    assert c["iters_total"] == T1 + T2a + T2b
    assert c["sigma"] == full["sigma"]
    assert np.array_equal(c["x_last"], full["x_last"])
    assert np.array_equal(xm, full["x_min"])
    assert c["t_min"] == full["t_min"] and c["L_min"] == full["L_min"]
    if mode == pa.SIGMA_MAX:  # sigma_max iterates are insensitive to round-off
        ro = oracle.projected_adam(A, mode, T1 + T2a + T2b, x_init=x0, **HYPER)
        assert np.linalg.norm(c["x_last"] - ro.x_last) <= 1e-10
        assert abs(c["sigma"] / ro.sigma - 1) <= 1e-10


def test_continue_full_size():
    """The 401 x 401 operator (964,806 rows, 304 CTAs): 20 + 20 = 40."""
    A = synth.hydro_operator(401, n_incl=8, eta_lo=1e18, eta_hi=1e24, seed=2)
    x0 = oracle.start_vector(A.n_cols, 1)
    with pa.create(A) as h:
        full = h.run(pa.SIGMA_MAX, 40, x0, **HYPER)
        h.run(pa.SIGMA_MAX, 20, x0, **HYPER)
        c = h.continue_run(20, **HYPER)
    assert c["sigma"] == full["sigma"]
    assert np.array_equal(c["x_last"], full["x_last"])


def test_continue_refuses_what_it_cannot_resume():
    A = synth.hydro_operator(13, seed=1)
    x0 = oracle.start_vector(A.n_cols, 1)
    with pa.create(A) as h:
        with pytest.raises(pa.PAError) as ei:  # nothing run yet
            h.continue_run(10, **HYPER)
        assert ei.value.status == -1
        h.run(pa.SIGMA_MAX, 10, x0, **HYPER)
        with pytest.raises(pa.PAError):  # other hyperparameters
            h.continue_run(10, lr=2e-2)
        h.continue_run(10, **HYPER)
    with pa.create(A, precision=pa.DF64) as h:  # the double-float kernel keeps no FP64 state
        h.run(pa.SIGMA_MAX, 10, x0, **HYPER)
        with pytest.raises(pa.PAError):
            h.continue_run(10, **HYPER)
