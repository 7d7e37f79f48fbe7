"""Matrices shared by the GPU parity test files (seeded, synthetic)."""
import numpy as np

from paper_2409_11515_gb300 import synth


def explicit_zeros():
    """A banded matrix plus explicit zeros: a fifth of its entries zeroed and
    one far-away zero per row (every stored zero must stay harmless, whatever
    the buffers it gathers from hold)."""
    A = synth.random_sparse(3000, 7, seed=11, diag_boost=4.0)
    rng = np.random.default_rng(12)
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    val = A.val.copy()
    off = rows != A.col
    val[off & (rng.random(A.nnz) < 0.2)] = 0.0
    far = (np.arange(A.n_rows) + A.n_rows // 2) % A.n_cols
    return synth.from_coo(np.concatenate([rows, np.arange(A.n_rows)]),
                          np.concatenate([A.col, far]),
                          np.concatenate([val, np.zeros(A.n_rows)]), A.n_rows, A.n_cols)


CASES = {
    "explicit_zeros": explicit_zeros,
    "hydro21": lambda: synth.hydro_operator(21, seed=1),
    "hydro13_8incl": lambda: synth.hydro_operator(13, 17, n_incl=8, seed=5),
    "lap2d_12": lambda: synth.laplacian_2d(12),
    "random_sparse": lambda: synth.random_sparse(3000, 9, seed=3, diag_boost=4.0),
    "rect_tall": lambda: synth.random_sparse(700, 5, seed=4, n_cols=500),
    "rect_wide": lambda: synth.random_sparse(300, 6, seed=6, n_cols=800),
}
