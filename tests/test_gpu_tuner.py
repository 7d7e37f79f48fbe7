"""The launch-shape tuner (autotune > 0): its choice is one of the variants it
timed, is recorded, is cached for later handles of the same matrix, and every
variant it can pick keeps the FP64 iterate parity with the oracle
(||x_t^gpu - x_t^cpu||_2 <= 1e-10 for t <= 100)."""
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


@pytest.fixture(scope="module")
def hydro81():
    # 39,366 rows: a grid of 19 CTAs, past the cluster engine's 16
    return synth.hydro_operator(81, seed=5)


@pytest.fixture(scope="module")
def reference(hydro81):
    x0 = oracle.start_vector(hydro81.n_cols, 2)
    return x0, oracle.projected_adam(hydro81, pa.SIGMA_MAX, 100, x_init=x0, n_trace=100,
                                     trace_L=True, **HYPER)


def test_choice_is_timed_recorded_and_cached(hydro81, reference):
    x0, ro = reference
    with pa.create(hydro81, autotune=2) as h:
        rg = h.run(pa.SIGMA_MAX, 100, x0, trace_L=True, n_trace=100, **HYPER)
        ch = h.launch_choice()
        info = h.last_run_info()
    assert ch["source"] == 1
    kinds = {(k, g) for k, g, _ in ch["trials"]}
    assert {0, 1, 6} <= {k for k, _ in kinds}  # three-phase, merged, single-pass
    assert (ch["kernel"], ch["grid"]) in kinds
    best = min(ch["trials"], key=lambda t: t[2])
    assert (ch["kernel"], ch["grid"]) == best[:2]
    assert (info["kernel"], info["grid"]) == (ch["kernel"], ch["grid"])
    assert np.max(np.linalg.norm(rg["x_trace"] - ro.x_trace, axis=1)) <= 1e-10
    with pa.create(hydro81, autotune=2) as h2:
        h2.run(pa.SIGMA_MAX, 30, x0, **HYPER)
        ch2 = h2.launch_choice()
        info2 = h2.last_run_info()
    assert ch2["source"] == 2 and ch2["trials"] == []
    assert (ch2["kernel"], ch2["grid"]) == (ch["kernel"], ch["grid"])
    assert (info2["kernel"], info2["grid"]) == (ch["kernel"], ch["grid"])


def test_untuned_handles_keep_the_default(hydro81, reference):
    x0, _ = reference
    with pa.create(hydro81) as h:
        h.run(pa.SIGMA_MAX, 30, x0, **HYPER)
        assert h.launch_choice()["kernel"] == -1
        assert h.last_run_info()["kernel"] == 0


@pytest.mark.parametrize("opt,kernel", [
    (dict(engine=pa.ENGINE_GRID), 0),
    (dict(engine=pa.ENGINE_GRID, grid_blocks=152), 0),  # one CTA per SM of a GB300
    (dict(engine=pa.ENGINE_MERGED), 1),
    (dict(engine=pa.ENGINE_SINGLE), 6),
], ids=["three_phase", "three_phase_1_per_sm", "merged", "single_pass"])
def test_every_candidate_keeps_parity(hydro81, reference, opt, kernel):
    x0, ro = reference
    with pa.create(hydro81, **opt) as h:
        rg = h.run(pa.SIGMA_MAX, 100, x0, trace_L=True, n_trace=100, **HYPER)
        assert h.last_run_info()["kernel"] == kernel
    assert np.max(np.linalg.norm(rg["x_trace"] - ro.x_trace, axis=1)) <= 1e-10
    Lo = ro.L_trace
    assert np.max(np.abs(rg["L_trace"] - Lo) / np.maximum(1, np.abs(Lo))) <= 1e-10
    assert rg["t_min"] == ro.t_min
