"""CPU oracle of the Projected Adam condition-number estimator.

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package.

The arithmetic lives in ``pa_oracle.c`` (plain serial FP64, compiled with
``-O2 -ffp-contract=off``); this module compiles it with gcc on first use and
marshals numpy arrays through ctypes.  It shares no code with the CUDA
library.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "pa_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liboracle.so"
_OMP_PATH = _BUILD / "liboracle_omp.so"
_lock = threading.Lock()
_lib = None

SIGMA_MAX, SIGMA_MIN = 1, 2
LOSS_LOGRATIO, LOSS_QUADRATIC = 0, 1
FLAG_DD, FLAG_NO_TANGENT, FLAG_NO_NORMALISE = 1, 2, 4
OK, SINGULAR, NONFINITE = 0, 1, -4


def build(force: bool = False, openmp: bool = False) -> Path:
    """Compile pa_oracle.c into oracle/_build/liboracle.so (gcc, -O2, no FMA
    contraction).  openmp=True builds liboracle_omp.so from the same source
    with -fopenmp: the same arithmetic with the loops on all host cores and
    per-thread partial sums -- for timing the oracle only, never as checker."""
    _BUILD.mkdir(exist_ok=True)
    out = _OMP_PATH if openmp else _LIB_PATH
    if not force and out.exists() and out.stat().st_mtime >= _SRC.stat().st_mtime:
        return out
    tmp = out.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC",
           *(["-fopenmp"] if openmp else []), str(_SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load_openmp() -> C.CDLL:
    """The OpenMP timing build (see build); use it through `using(...)`."""
    return load(build(openmp=True))


def load(path) -> C.CDLL:
    """Load a compiled copy of pa_oracle.c (the default build or a test's variant)."""
    L = C.CDLL(str(path))
    _declare(L)
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


_active = threading.local()


def _L():
    return getattr(_active, "lib", None) or lib()


class using:
    """Context manager: route the module functions through another compiled copy."""

    def __init__(self, L):
        self.L = L

    def __enter__(self):
        self.prev = getattr(_active, "lib", None)
        _active.lib = self.L
        return self.L

    def __exit__(self, *exc):
        _active.lib = self.prev


def compile_variant(source_text: str, out_path, contract_fma: bool = False) -> Path:
    """Compile an edited copy of the oracle source (mutation tests), or the
    unchanged source with fused multiply-add contraction (contract_fma): the
    same algorithm under a different rounding, used to measure how strongly
    an iteration amplifies round-off."""
    out_path = Path(out_path)
    src = out_path.with_suffix(".c")
    src.write_text(source_text)
    flags = ["-ffp-contract=fast"] if contract_fma else ["-ffp-contract=off"]
    if contract_fma and platform.machine() in ("x86_64", "AMD64"):
        flags.append("-mfma")  # aarch64 has FMA in its base ISA
    subprocess.run(["gcc", "-O2", *flags, "-fno-fast-math", "-std=c11", "-shared",
                    "-fPIC", str(src), "-o", str(out_path), "-lm"], check=True)
    return out_path


def rounding_ensemble(A, mode: int, iters: int, x_init, workdir, loss: int = LOSS_LOGRATIO,
                      n_perturbed: int = 2, n_entries: int = 3, flags: int = 0, **hyper):
    """Runs of the same Algorithm 1 that differ from the oracle only in
    round-off: the FMA-contracted build of this source, and x_init with a few
    entries moved by one ulp.  Returns (reference run, [variant runs])."""
    x_init = np.ascontiguousarray(x_init, dtype=np.float64)
    ref = projected_adam(A, mode, iters, x_init=x_init, loss=loss, n_trace=iters, trace_L=True,
                         flags=flags, **hyper)
    runs = []
    fma = load(compile_variant(source_text(), Path(workdir) / "oracle_fma.so", contract_fma=True))
    with using(fma):
        runs.append(projected_adam(A, mode, iters, x_init=x_init, loss=loss, n_trace=iters,
                                   trace_L=True, flags=flags, **hyper))
    rng = np.random.default_rng(12345)
    for _ in range(n_perturbed):
        xp = x_init.copy()
        idx = rng.choice(xp.size, size=min(n_entries, xp.size), replace=False)
        xp[idx] = np.nextafter(xp[idx], np.inf)
        runs.append(projected_adam(A, mode, iters, x_init=xp, loss=loss, n_trace=iters,
                                   trace_L=True, flags=flags, **hyper))
    return ref, runs


def source_text() -> str:
    return _SRC.read_text()


def _declare(L):
    d, i32, i64, u64, p = C.c_double, C.c_int32, C.c_int64, C.c_uint64, C.c_void_p
    L.po_splitmix64_at.restype = u64
    L.po_splitmix64_at.argtypes = [u64, u64]
    L.po_start_vector.restype = None
    L.po_start_vector.argtypes = [i64, u64, p]
    L.po_spmv.restype = None
    L.po_spmv.argtypes = [i32, p, p, p, p, p]
    L.po_spmv_t.restype = None
    L.po_spmv_t.argtypes = [i32, i32, p, p, p, p, p]
    L.po_spmv_dd.restype = None
    L.po_spmv_dd.argtypes = [i32, p, p, p, p, p, p]
    L.po_spmv_t_dd.restype = None
    L.po_spmv_t_dd.argtypes = [i32, i32, p, p, p, p, p, p]
    L.po_projected_adam.restype = C.c_int
    L.po_projected_adam.argtypes = [i32, i32, p, p, p, C.c_int, C.c_int, i64, d, d, d, d,
                                    p, C.c_int, p, p, p, p, p, i64]
    L.po_sigma.restype = d
    L.po_sigma.argtypes = [i32, i32, p, p, p, p, C.c_int]
    L.po_loss_grad.restype = d
    L.po_loss_grad.argtypes = [i32, i32, p, p, p, C.c_int, C.c_int, p, p]
    L.po_equilibrate_pow2.restype = None
    L.po_equilibrate_pow2.argtypes = [i32, i32, p, p, p, p, p, p]
    L.po_error_bounds.restype = None
    L.po_error_bounds.argtypes = [i32, i32, p, p, p, p, p, d, d, d, p]
    for name in ("po_lower_solve", "po_upper_solve", "po_upper_t_solve", "po_lower_t_solve"):
        getattr(L, name).restype = None
        getattr(L, name).argtypes = [i32, p, p, p, p, p]
    L.po_lu_products.restype = None
    L.po_lu_products.argtypes = [i32, p, p, p, p, p, p, p, p, p, p, p]
    L.po_projected_adam_lu.restype = C.c_int
    L.po_projected_adam_lu.argtypes = [i32, p, p, p, p, p, p, p, p, i64, d, d, d, d, p, p, p, p,
                                       p, p, i64]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _csr(A):
    row_ptr, col, val, n_rows, n_cols = A.astuple() if hasattr(A, "astuple") else A
    return (np.ascontiguousarray(row_ptr, dtype=np.int32), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64), int(n_rows), int(n_cols))


def splitmix64_at(seed: int, i: int) -> int:
    return int(_L().po_splitmix64_at(seed & (2**64 - 1), i))


def start_vector(n: int, seed: int) -> np.ndarray:
    x = np.empty(n, dtype=np.float64)
    _L().po_start_vector(n, seed & (2**64 - 1), _ptr(x))
    return x


def spmv(A, x, dd: bool = False):
    rp, ci, va, m, n = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(m, dtype=np.float64)
    if dd:
        ylo = np.empty(m, dtype=np.float64)
        _L().po_spmv_dd(m, _ptr(rp), _ptr(ci), _ptr(va), _ptr(x), _ptr(y), _ptr(ylo))
        return y, ylo
    _L().po_spmv(m, _ptr(rp), _ptr(ci), _ptr(va), _ptr(x), _ptr(y))
    return y


def spmv_t(A, y, y_lo=None):
    rp, ci, va, m, n = _csr(A)
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.empty(n, dtype=np.float64)
    if y_lo is not None:
        y_lo = np.ascontiguousarray(y_lo, dtype=np.float64)
        _L().po_spmv_t_dd(m, n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(y), _ptr(y_lo), _ptr(z))
    else:
        _L().po_spmv_t(m, n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(y), _ptr(z))
    return z


def sigma(A, x, dd: bool = False) -> float:
    rp, ci, va, m, n = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(_L().po_sigma(m, n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(x), FLAG_DD if dd else 0))


def loss_grad(A, x, mode: int, loss: int = LOSS_LOGRATIO):
    """(L(x), grad L(x)) of Eq. nabla_loss (negated for sigma_min)."""
    rp, ci, va, m, n = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.empty(n, dtype=np.float64)
    L = _L().po_loss_grad(m, n, _ptr(rp), _ptr(ci), _ptr(va), mode, loss, _ptr(x), _ptr(g))
    return float(L), g


def equilibrate_pow2(A):
    rp, ci, va, m, n = _csr(A)
    dr = np.empty(m, dtype=np.float64)
    dc = np.empty(n, dtype=np.float64)
    vh = np.empty(va.size, dtype=np.float64)
    _L().po_equilibrate_pow2(m, n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(dr), _ptr(dc), _ptr(vh))
    return dr, dc, vh


ERROR_BOUND_KEYS = ("residual_norm", "b_norm", "x_hat_norm", "thm1_lower", "thm1_upper",
                    "thm2_lower", "thm2_upper", "thm3_upper", "thm4_rounding", "singular")


def error_bounds(A, x_hat, b, kappa: float, norm_a: float, u: float = 2.0 ** -53) -> dict:
    """Residual (Dot2) of x_hat for A x = b and the bounds of the paper's
    Theorems 1-4 (po_error_bounds)."""
    rp, ci, va, m, n = _csr(A)
    x_hat = np.ascontiguousarray(x_hat, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.empty(10)
    _L().po_error_bounds(m, n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(x_hat), _ptr(b), kappa, norm_a,
                         u, _ptr(out))
    return dict(zip(ERROR_BOUND_KEYS, out.tolist()))


def triangular_solve(T, b, kind: str) -> np.ndarray:
    """kind: 'lower' (T x = b), 'upper', 'upper_t' (T^T x = b, T upper) or
    'lower_t' (T^T x = b, T lower); T in CSR with its diagonal stored."""
    rp, ci, va, n, _ = _csr(T)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(n)
    getattr(_L(), f"po_{kind}_solve")(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(b), _ptr(x))
    return x


def _perm(p, n):
    return None if p is None else np.ascontiguousarray(p, dtype=np.int32)


def lu_products(Lf, Uf, p, q, x):
    """(r, s) = (A^{-1} x, A^{-T} A^{-1} x) for P A Q = L U (Algorithm 2's solves)."""
    lrp, lci, lva, n, _ = _csr(Lf)
    urp, uci, uva, _, _ = _csr(Uf)
    p, q = _perm(p, n), _perm(q, n)
    x = np.ascontiguousarray(x, dtype=np.float64)
    r, s = np.empty(n), np.empty(n)
    _L().po_lu_products(n, _ptr(lrp), _ptr(lci), _ptr(lva), _ptr(urp), _ptr(uci), _ptr(uva),
                        _ptr(p), _ptr(q), _ptr(x), _ptr(r), _ptr(s))
    return r, s


def projected_adam_lu(Lf, Uf, p, q, iters: int, x_init, lr: float = 1e-2, beta1: float = 0.9,
                      beta2: float = 0.999, eps: float = 1e-12, n_trace: int = 0,
                      trace_L: bool = False):
    """Algorithm 1 on A^{-1} with Algorithm 2's gradient; sigma_min = 1 / sigma."""
    lrp, lci, lva, n, _ = _csr(Lf)
    urp, uci, uva, _, _ = _csr(Uf)
    p, q = _perm(p, n), _perm(q, n)
    x_init = np.ascontiguousarray(x_init, dtype=np.float64)
    x_min, x_last, out = np.empty(n), np.empty(n), np.empty(5)
    L_trace = np.empty(iters) if trace_L else None
    x_trace = np.empty((n_trace, n)) if n_trace else None
    st = _L().po_projected_adam_lu(n, _ptr(lrp), _ptr(lci), _ptr(lva), _ptr(urp), _ptr(uci),
                                   _ptr(uva), _ptr(p), _ptr(q), iters, lr, beta1, beta2, eps,
                                   _ptr(x_init), _ptr(x_min), _ptr(x_last), _ptr(out),
                                   _ptr(L_trace), _ptr(x_trace), n_trace)
    return AdamResult(status=st, x_min=x_min, x_last=x_last, L_min=out[0], t_min=int(out[1]),
                      L_last=out[2], iters_run=int(out[3]), sigma=out[4], sigma_min=1.0 / out[4],
                      L_trace=L_trace, x_trace=x_trace)


class AdamResult(dict):
    __getattr__ = dict.__getitem__


def projected_adam(A, mode: int, iters: int, lr: float = 1e-2, beta1: float = 0.9,
                   beta2: float = 0.999, eps: float = 1e-12, x_init=None, seed: int | None = None,
                   loss: int = LOSS_LOGRATIO, flags: int = 0, n_trace: int = 0,
                   trace_L: bool = False) -> AdamResult:
    """Algorithm 1 (Projected Adam) on A for sigma_max (mode=1) or sigma_min (mode=2)."""
    rp, ci, va, m, n = _csr(A)
    if x_init is None:
        x_init = start_vector(n, 1 if seed is None else seed)
    x_init = np.ascontiguousarray(x_init, dtype=np.float64)
    x_min = np.empty(n)
    x_last = np.empty(n)
    out = np.empty(4)
    L_trace = np.empty(iters) if trace_L else None
    x_trace = np.empty((n_trace, n)) if n_trace > 0 else None
    st = _L().po_projected_adam(m, n, _ptr(rp), _ptr(ci), _ptr(va), mode, loss, iters, lr, beta1,
                                 beta2, eps, _ptr(x_init), flags, _ptr(x_min), _ptr(x_last),
                                 _ptr(out), _ptr(L_trace), _ptr(x_trace), n_trace)
    sig = sigma(A, x_min, dd=bool(flags & FLAG_DD))
    return AdamResult(status=int(st), x_min=x_min, x_last=x_last, L_min=out[0], t_min=int(out[1]),
                      L_last=out[2], iters_run=int(out[3]), L_trace=L_trace, x_trace=x_trace,
                      sigma=sig)


def estimate(A, iters_max: int, iters_min: int, seed: int = 1, lr: float = 1e-2,
             beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-12,
             loss: int = LOSS_LOGRATIO, flags_min: int = 0):
    """kappa_2 = sigma_max / sigma_min, both from Algorithm 1 with the same x_init."""
    n = _csr(A)[4]
    x0 = start_vector(n, seed)
    rmax = projected_adam(A, SIGMA_MAX, iters_max, lr, beta1, beta2, eps, x_init=x0, loss=loss)
    rmin = projected_adam(A, SIGMA_MIN, iters_min, lr, beta1, beta2, eps, x_init=x0, loss=loss,
                          flags=flags_min)
    smax, smin = rmax.sigma, rmin.sigma
    kappa = smax / smin if smin > 0 else float("inf")
    return dict(sigma_max=smax, sigma_min=smin, kappa=kappa, status_max=rmax.status,
                status_min=rmin.status, max=rmax, min=rmin)
