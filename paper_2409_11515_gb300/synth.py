"""Seeded synthetic inputs: sparse matrices in int32 CSR with float64 values.

This module only builds test and benchmark operators. It holds none of the
Projected Adam arithmetic (no SpMV, no Adam step, no norm, no start vector),
so both the CPU oracle and the CUDA path can take their matrices from here
without sharing any of the method's code.

Operators
---------
* ``diag_csr``         diagonal matrix, singular values = |d_i|.
* ``laplacian_1d``     tridiag(-1, 2, -1), Dirichlet, n points.
* ``laplacian_2d``     5-point Dirichlet Laplacian on an N x N grid.
* ``dense_csr``        a dense matrix stored as CSR (every entry present).
* ``random_sparse``    seeded random pattern with a fixed count per row.
* ``hydro_operator``   stand-in for the paper's benchmark systems: the
  2D staggered-grid hydro-mechanical (Stokes + Darcy, Biot-coupled) operator
  of the paper's benchmark model section (governing equations, marker-in-cell
  discretisation). The paper's own 360960 x 360960 matrices are not
  available, so this generator reproduces their structure instead: six
  interleaved unknowns per cell, a tri-banded pattern, about 7 non-zeros per
  row, and column norms split into a small group (pressures, < 1e-2) and a
  large group (velocities and Darcy fluxes, > 1e10), as the paper's
  column-norm figure describes.
* ``hydro_batch``      many hydro operators with seeded, uneven grid sizes.

Every function returns ``(row_ptr, col, val, n_rows, n_cols)`` with
``row_ptr`` int32[n_rows+1], ``col`` int32[nnz] (sorted within each row, no
duplicates), ``val`` float64[nnz].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR", "diag_csr", "laplacian_1d", "laplacian_2d", "dense_csr", "random_sparse",
    "hydro_operator", "hydro_batch", "HYDRO_FIELDS", "csr_to_dense", "from_coo",
]

HYDRO_FIELDS = ("vx", "vy", "P", "qx", "qy", "Pf")


@dataclass
class CSR:
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    n_rows: int
    n_cols: int

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def astuple(self):
        return self.row_ptr, self.col, self.val, self.n_rows, self.n_cols


def from_coo(rows, cols, vals, n_rows, n_cols) -> CSR:
    """Sort triplets by (row, col) and pack them as CSR (no duplicate merge)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n_rows)
    row_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz does not fit int32 CSR")
    return CSR(row_ptr.astype(np.int32), cols.astype(np.int32),
               np.ascontiguousarray(vals), int(n_rows), int(n_cols))


def csr_to_dense(A: CSR) -> np.ndarray:
    D = np.zeros((A.n_rows, A.n_cols), dtype=np.float64)
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr.astype(np.int64)))
    np.add.at(D, (rows, A.col.astype(np.int64)), A.val)
    return D


def diag_csr(d) -> CSR:
    d = np.asarray(d, dtype=np.float64)
    n = d.size
    return CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d.copy(), n, n)


def laplacian_1d(n: int) -> CSR:
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[1:] - 1, i[:-1] + 1])
    vals = np.concatenate([np.full(n, 2.0), np.full(n - 1, -1.0), np.full(n - 1, -1.0)])
    return from_coo(rows, cols, vals, n, n)


def laplacian_2d(N: int) -> CSR:
    """5-point Laplacian, Dirichlet, unknown (i, j) at index j*N + i."""
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    k = jj * N + ii
    rows, cols, vals = [k], [k], [np.full(k.size, 4.0)]
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        ok = (ii + di >= 0) & (ii + di < N) & (jj + dj >= 0) & (jj + dj < N)
        rows.append(k[ok])
        cols.append((jj[ok] + dj) * N + ii[ok] + di)
        vals.append(np.full(int(ok.sum()), -1.0))
    return from_coo(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), N * N, N * N)


def dense_csr(M) -> CSR:
    M = np.asarray(M, dtype=np.float64)
    m, n = M.shape
    rr, cc = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    return from_coo(rr.ravel(), cc.ravel(), M.ravel(), m, n)


def random_sparse(n: int, per_row: int, seed: int, n_cols: int | None = None,
                  diag_boost: float = 0.0, band: int | None = None) -> CSR:
    """Seeded random pattern: ``per_row`` distinct columns per row, N(0,1) values.

    ``band`` restricts columns to |j - i| <= band (wrapped into range);
    ``diag_boost`` adds a diagonal entry of that size (square only).
    """
    n_cols = n if n_cols is None else n_cols
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        if band is None:
            c = rng.choice(n_cols, size=min(per_row, n_cols), replace=False)
        else:
            lo, hi = max(0, i - band), min(n_cols, i + band + 1)
            c = rng.choice(np.arange(lo, hi), size=min(per_row, hi - lo), replace=False)
        rows.append(np.full(c.size, i))
        cols.append(c)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = rng.standard_normal(rows.size)
    if diag_boost:
        key = rows * n_cols + cols
        d = np.arange(min(n, n_cols))
        dkey = d * n_cols + d
        present = np.isin(dkey, key)
        vals[np.isin(key, dkey)] += diag_boost
        rows = np.concatenate([rows, d[~present]])
        cols = np.concatenate([cols, d[~present]])
        vals = np.concatenate([vals, np.full(int((~present).sum()), diag_boost)])
    return from_coo(rows, cols, vals, n, n_cols)


# ----------------------------------------------------------------------------
# Hydro-mechanical staggered-grid operator
# ----------------------------------------------------------------------------

@dataclass
class HydroParams:
    nx: int
    ny: int
    dx: float = 500.0
    dy: float = 500.0
    n_incl: int = 4
    eta_bg: float = 1e21           # solid shear viscosity of the matrix (Pa s)
    eta_lo: float = 1e18           # inclusion viscosity, log-uniform in [lo, hi]
    eta_hi: float = 1e24
    keta_lo: float = 1e-20         # k / eta_fluid, per cell, log-uniform
    keta_hi: float = 1e-12
    phi: float = 0.01              # porosity
    alpha: float = 0.9             # Biot-Willis coefficient
    skempton: float = 0.6          # B
    beta_d: float = 1e-11          # drained compressibility (1/Pa)
    dt: float = 1e10               # time step (s)
    seed: int = 1


def _material_fields(p: HydroParams):
    rng = np.random.default_rng(p.seed)
    W, H = p.nx * p.dx, p.ny * p.dy
    cx = rng.uniform(0.1 * W, 0.9 * W, p.n_incl)
    cy = rng.uniform(0.1 * H, 0.9 * H, p.n_incl)
    rad = rng.uniform(0.05, 0.15, p.n_incl) * min(W, H)
    eta_in = np.exp(rng.uniform(math.log(p.eta_lo), math.log(p.eta_hi), p.n_incl))
    keta = np.exp(rng.uniform(math.log(p.keta_lo), math.log(p.keta_hi), (p.ny, p.nx)))

    def eta_at(X, Y):
        e = np.full(X.shape, p.eta_bg)
        for c in range(p.n_incl):  # later inclusions overwrite earlier ones
            inside = (X - cx[c]) ** 2 + (Y - cy[c]) ** 2 <= rad[c] ** 2
            e[inside] = eta_in[c]
        return e

    jj, ii = np.meshgrid(np.arange(p.ny), np.arange(p.nx), indexing="ij")
    eta_c = eta_at((ii + 0.5) * p.dx, (jj + 0.5) * p.dy)   # cell centres
    eta_n = eta_at(ii * p.dx, jj * p.dy)                   # basic (corner) nodes
    return eta_c, eta_n, keta


def hydro_operator(nx: int, ny: int | None = None, *, n_incl: int = 4, eta_lo: float = 1e18,
                   eta_hi: float = 1e24, keta_lo: float = 1e-20, keta_hi: float = 1e-12,
                   seed: int = 1, dx: float = 500.0, dy: float = 500.0) -> CSR:
    """Assemble the 6-unknown-per-cell hydro-mechanical operator on an nx x ny grid.

    Index of unknown f of cell (i, j): 6*(j*nx + i) + f with f in
    (vx, vy, P, qx, qy, Pf).  n = 6*nx*ny.  Positions on the staggered grid:
    vx, qx on x-faces (i*dx, (j+1/2)*dy); vy, qy on y-faces ((i+1/2)*dx, j*dy);
    P, Pf at cell centres.  The last column/row of cells is a ghost layer.

    Rows (interior):
      x/y momentum  : variable-viscosity normal + shear stress divergence
                      (5 own-component + 4 cross-component entries) minus the
                      pressure gradient (2 entries) = 11 entries; free slip on
                      the walls parallel to the component.
      solid mass    : div(v) + beta_d/dt (P - alpha Pf) + (P - Pf)/((1-phi) eta_phi)
                      = 6 entries.
      Darcy x/y     : (eta_f/k) q + grad Pf = 3 entries.
      fluid mass    : div(q) - beta_d alpha/dt (P - Pf/B) - (P - Pf)/((1-phi) eta_phi)
                      = 6 entries.
    Dirichlet velocities, no-flux Darcy boundaries, ghost unknowns and one
    pinned P and Pf cell are identity rows.
    """
    ny = nx if ny is None else ny
    if nx < 3 or ny < 3:
        raise ValueError("hydro_operator needs nx, ny >= 3")
    p = HydroParams(nx=nx, ny=ny, dx=dx, dy=dy, n_incl=n_incl, eta_lo=eta_lo, eta_hi=eta_hi,
                    keta_lo=keta_lo, keta_hi=keta_hi, seed=seed)
    eta_c, eta_n, keta = _material_fields(p)
    n = 6 * nx * ny
    VX, VY, P, QX, QY, PF = range(6)

    def idx(i, j, f):
        return 6 * (j * nx + i) + f

    R, C, V = [], [], []

    def add(rows, cols, vals):
        rows = np.broadcast_to(rows, np.broadcast(rows, cols, vals).shape)
        R.append(np.asarray(rows).ravel())
        C.append(np.broadcast_to(cols, rows.shape).ravel())
        V.append(np.broadcast_to(vals, rows.shape).astype(np.float64).ravel())

    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    dx2, dy2, dxdy = dx * dx, dy * dy, dx * dy

    # ---- x-momentum at vx(i, j), 1 <= i <= nx-2, 0 <= j <= ny-2
    m = (ii >= 1) & (ii <= nx - 2) & (jj <= ny - 2)
    i, j = ii[m], jj[m]
    r = idx(i, j, VX)
    ec_r, ec_l = eta_c[j, i], eta_c[j, i - 1]
    top = j <= ny - 3            # shear term at node row j+1 is interior
    bot = j >= 1                 # shear term at node row j is interior
    en_t = np.where(top, eta_n[np.minimum(j + 1, ny - 1), i], 0.0)
    en_b = np.where(bot, eta_n[j, i], 0.0)
    add(r, idx(i + 1, j, VX), 2 * ec_r / dx2)
    add(r, idx(i - 1, j, VX), 2 * ec_l / dx2)
    add(r, idx(i, j, VX), -2 * (ec_r + ec_l) / dx2 - (en_t + en_b) / dy2)
    t = top
    add(r[t], idx(i[t], j[t] + 1, VX), en_t[t] / dy2)
    add(r[t], idx(i[t], j[t] + 1, VY), en_t[t] / dxdy)
    add(r[t], idx(i[t] - 1, j[t] + 1, VY), -en_t[t] / dxdy)
    b = bot
    add(r[b], idx(i[b], j[b] - 1, VX), en_b[b] / dy2)
    add(r[b], idx(i[b], j[b], VY), -en_b[b] / dxdy)
    add(r[b], idx(i[b] - 1, j[b], VY), en_b[b] / dxdy)
    add(r, idx(i, j, P), -1.0 / dx)
    add(r, idx(i - 1, j, P), 1.0 / dx)

    # ---- y-momentum at vy(i, j), 0 <= i <= nx-2, 1 <= j <= ny-2
    m = (jj >= 1) & (jj <= ny - 2) & (ii <= nx - 2)
    i, j = ii[m], jj[m]
    r = idx(i, j, VY)
    ec_u, ec_d = eta_c[j, i], eta_c[j - 1, i]
    rgt = i <= nx - 3
    lft = i >= 1
    en_r = np.where(rgt, eta_n[j, np.minimum(i + 1, nx - 1)], 0.0)
    en_l = np.where(lft, eta_n[j, i], 0.0)
    add(r, idx(i, j + 1, VY), 2 * ec_u / dy2)
    add(r, idx(i, j - 1, VY), 2 * ec_d / dy2)
    add(r, idx(i, j, VY), -2 * (ec_u + ec_d) / dy2 - (en_r + en_l) / dx2)
    t = rgt
    add(r[t], idx(i[t] + 1, j[t], VY), en_r[t] / dx2)
    add(r[t], idx(i[t] + 1, j[t], VX), en_r[t] / dxdy)
    add(r[t], idx(i[t] + 1, j[t] - 1, VX), -en_r[t] / dxdy)
    t = lft
    add(r[t], idx(i[t] - 1, j[t], VY), en_l[t] / dx2)
    add(r[t], idx(i[t], j[t], VX), -en_l[t] / dxdy)
    add(r[t], idx(i[t], j[t] - 1, VX), en_l[t] / dxdy)
    add(r, idx(i, j, P), -1.0 / dy)
    add(r, idx(i, j - 1, P), 1.0 / dy)

    # ---- cell-centred rows, 0 <= i <= nx-2, 0 <= j <= ny-2, (0, 0) pinned.
    # Both mass equations are multiplied by kc = eta_bg/dx, the usual
    # geodynamic balancing of continuity rows against momentum rows; the
    # pressure unknowns themselves stay unscaled, so their columns stay small.
    m = (ii <= nx - 2) & (jj <= ny - 2) & ~((ii == 0) & (jj == 0))
    i, j = ii[m], jj[m]
    eta_phi = eta_c[j, i] / p.phi
    comp = 1.0 / ((1.0 - p.phi) * eta_phi)
    bd = p.beta_d / p.dt
    kc = p.eta_bg / dx
    # solid mass
    r = idx(i, j, P)
    add(r, idx(i + 1, j, VX), kc / dx)
    add(r, idx(i, j, VX), -kc / dx)
    add(r, idx(i, j + 1, VY), kc / dy)
    add(r, idx(i, j, VY), -kc / dy)
    add(r, idx(i, j, P), kc * (bd + comp))
    add(r, idx(i, j, PF), -kc * (p.alpha * bd + comp))
    # fluid mass
    r = idx(i, j, PF)
    add(r, idx(i + 1, j, QX), kc / dx)
    add(r, idx(i, j, QX), -kc / dx)
    add(r, idx(i, j + 1, QY), kc / dy)
    add(r, idx(i, j, QY), -kc / dy)
    add(r, idx(i, j, P), -kc * (p.alpha * bd + comp))
    add(r, idx(i, j, PF), kc * (p.alpha * bd / p.skempton + comp))

    # ---- Darcy x at qx(i, j), 1 <= i <= nx-2, 0 <= j <= ny-2
    m = (ii >= 1) & (ii <= nx - 2) & (jj <= ny - 2)
    i, j = ii[m], jj[m]
    r = idx(i, j, QX)
    kf = 0.5 * (keta[j, i] + keta[j, i - 1])
    add(r, r, 1.0 / kf)
    add(r, idx(i, j, PF), 1.0 / dx)
    add(r, idx(i - 1, j, PF), -1.0 / dx)
    # ---- Darcy y at qy(i, j), 0 <= i <= nx-2, 1 <= j <= ny-2
    m = (jj >= 1) & (jj <= ny - 2) & (ii <= nx - 2)
    i, j = ii[m], jj[m]
    r = idx(i, j, QY)
    kf = 0.5 * (keta[j, i] + keta[j - 1, i])
    add(r, r, 1.0 / kf)
    add(r, idx(i, j, PF), 1.0 / dy)
    add(r, idx(i, j - 1, PF), -1.0 / dy)

    # ---- identity rows for every unknown that has no equation above, each
    # weighted like the diagonal of its field's equations (kbond): velocities
    # by 4 eta_bg/dx^2, Darcy fluxes by the mean eta_f/k, pressures by 1/dx.
    have = np.zeros(n, dtype=bool)
    for rr in R:
        have[rr] = True
    ident = np.nonzero(~have)[0]
    f = ident % 6
    kb = np.array([4 * p.eta_bg / dx2, 4 * p.eta_bg / dx2, 1.0 / dx,
                   1.0 / math.sqrt(p.keta_lo * p.keta_hi), 1.0 / math.sqrt(p.keta_lo * p.keta_hi),
                   1.0 / dx])
    add(ident, ident, kb[f])

    A = from_coo(np.concatenate(R), np.concatenate(C), np.concatenate(V), n, n)
    # the stencils above never place two entries at the same (row, col)
    return A


def hydro_batch(n_mat: int, lo: int, hi: int, seed: int, **kw) -> list[CSR]:
    """``n_mat`` hydro operators with grid side drawn uniformly from [lo, hi]."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, size=(n_mat, 2))
    return [hydro_operator(int(a), int(b), seed=seed * 1000 + k, **kw)
            for k, (a, b) in enumerate(sides)]
