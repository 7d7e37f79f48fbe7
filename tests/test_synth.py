"""Generator checks: determinism, CSR validity and the paper's matrix statistics."""
import hashlib

import numpy as np
import pytest

from paper_2409_11515_gb300 import synth


def _digest(A):
    h = hashlib.sha256()
    for a in (A.row_ptr, A.col, A.val):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _valid(A):
    assert A.row_ptr.dtype == np.int32 and A.col.dtype == np.int32 and A.val.dtype == np.float64
    assert A.row_ptr[0] == 0 and A.row_ptr[-1] == A.val.size == A.col.size
    assert np.all(np.diff(A.row_ptr) >= 0)
    assert A.col.min() >= 0 and A.col.max() < A.n_cols
    for i in range(0, A.n_rows, max(1, A.n_rows // 200)):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)  # sorted, no duplicates


def test_hydro_deterministic_and_valid():
    a, b = synth.hydro_operator(21, seed=1), synth.hydro_operator(21, seed=1)
    assert _digest(a) == _digest(b)
    assert _digest(a) != _digest(synth.hydro_operator(21, seed=2))
    _valid(a)
    assert a.n_rows == 6 * 21 * 21 == 2646


@pytest.mark.parametrize("nx", [21, 61])
def test_hydro_matches_paper_statistics(nx):
    A = synth.hydro_operator(nx, seed=1)
    per_row = A.nnz / A.n_rows
    # the paper's matrix: 2,575,716 nnz / 360,960 rows = 7.14 per row
    assert 5.5 < per_row < 7.2
    assert np.max(np.diff(A.row_ptr)) == 11
    cn = np.sqrt(np.bincount(A.col, weights=A.val ** 2, minlength=A.n_cols))
    small, large = np.mean(cn < 1e-2), np.mean(cn > 1e10)
    # the paper: 32.4 % of columns below 1e-2, 67.6 % above 1e10
    assert 0.28 < small < 0.36 and 0.6 < large < 0.7
    # tri-banded: every entry within 6*(nx+1) of the diagonal
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    assert np.max(np.abs(A.col - rows)) <= 6 * (nx + 1)


def test_hydro_conditioning_like_the_paper():
    # kappa(A) beyond 1/eps and column scaling cutting it by many orders
    A = synth.hydro_operator(21, seed=1)
    M = synth.csr_to_dense(A)
    cn = np.linalg.norm(M, axis=0)
    s = np.linalg.svd(M / cn, compute_uv=False)
    kappa_scaled = s[0] / s[-1]
    smax = np.linalg.svd(M, compute_uv=False)[0]
    smin = 1.0 / np.linalg.norm(np.linalg.inv(M / cn) / cn[:, None], 2)
    assert smax / smin > 1e20
    assert kappa_scaled < 1e7


def test_small_generators():
    _valid(synth.laplacian_1d(9))
    _valid(synth.laplacian_2d(5))
    _valid(synth.random_sparse(50, 4, seed=1, diag_boost=2.0))
    _valid(synth.random_sparse(30, 3, seed=2, band=5))
    M = np.arange(12.0).reshape(3, 4) - 5
    assert np.array_equal(synth.csr_to_dense(synth.dense_csr(M)), M)
    batch = synth.hydro_batch(4, 5, 9, seed=3)
    assert len(batch) == 4 and all(b.n_rows % 6 == 0 for b in batch)
