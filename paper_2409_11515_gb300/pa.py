"""Python binding of libpa (include/pa.h): argument marshalling only.

Every computation happens in the library's CUDA kernels.  PyTorch supplies
device memory (through the allocator hooks of pa_set_allocator) and streams.
The binding raises ``LibraryMissing`` when ``_build/libpa.so`` has not been
built: there is no CPU fallback.

Names follow the C ABI: ``create`` (pa_create), ``Handle.estimate``
(pa_estimate), ``Handle.run`` (pa_run), ``estimate_batched``
(pa_estimate_batched), ``Handle.get_vector``, ``Handle.spmv``,
``Handle.spmv_t``, ``Handle.get_transpose``, ``Handle.destroy``.
"""
from __future__ import annotations

import ctypes as C
import threading
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_build" / "libpa.so"

SIGMA_MAX, SIGMA_MIN, BOTH, SIGMA_MIN_LU, BOTH_LU = 1, 2, 3, 4, 5
HOST, DEVICE = 0, 1
LOSS_LOGRATIO, LOSS_QUADRATIC = 0, 1
FP64, MIXED, DF64 = 0, 1, 2
EQ_NONE, EQ_STORAGE, EQ_TARGET = 0, 1, 2
ENGINE_AUTO, ENGINE_GRID, ENGINE_CLUSTER, ENGINE_MERGED, ENGINE_SINGLE = 0, 1, 2, 3, 4
ABLATE_NO_TANGENT, ABLATE_NO_NORMALISE = 1, 2

OK, WARN_SINGULAR = 0, 1
STATUS_NAMES = {0: "PA_OK", 1: "PA_WARN_SINGULAR", -1: "PA_ERR_INVALID_ARG",
                -2: "PA_ERR_INVALID_CSR", -3: "PA_ERR_NOT_SQUARE", -4: "PA_ERR_NONFINITE",
                -5: "PA_ERR_TIMEOUT", -6: "PA_ERR_CUDA", -7: "PA_ERR_OOM", -8: "PA_ERR_LAUNCH",
                -9: "PA_ERR_UNSUPPORTED"}

EXPORTS = ("pa_options_default", "pa_create", "pa_estimate", "pa_run", "pa_estimate_batched",
           "pa_get_vector", "pa_spmv", "pa_spmv_t", "pa_get_transpose", "pa_get_equilibration",
           "pa_kernel_launches", "pa_destroy", "pa_last_error", "pa_set_allocator",
           "pa_last_run_profile", "pa_last_run_info", "pa_continue", "pa_sigma_noalloc", "pa_last_batch_graph", "pa_error_bounds", "pa_attach_lu",
           "pa_spmv_ata", "pa_single_pass_info", "pa_launch_choice", "pa_lu_route_info")

ERROR_BOUND_KEYS = ("residual_norm", "b_norm", "x_hat_norm", "thm1_lower", "thm1_upper",
                    "thm2_lower", "thm2_upper", "thm3_upper", "thm4_rounding", "singular")


class LibraryMissing(RuntimeError):
    pass


class PAError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("loss", C.c_int), ("precision", C.c_int), ("equilibrate", C.c_int),
                ("engine", C.c_int), ("ablation", C.c_int), ("barrier_timeout_ns", C.c_int64),
                ("grid_blocks", C.c_int), ("debug_skip_arrival", C.c_int),
                ("fp64_tail", C.c_int), ("autotune", C.c_int)]


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lib = None
_lock = threading.Lock()
_hooks = None


def load(path: Path | str | None = None):
    """Load libpa.so (building is ``paper_2409_11515_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = Path(path) if path else LIB_PATH
        if not p.exists():
            raise LibraryMissing(f"{p} is not built; run paper_2409_11515_gb300.build.build()")
        L = C.CDLL(str(p))
        _declare(L)
        if path is None:
            _lib = L
        return L


def _declare(L):
    i32, i64, u64, d, vp = C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_void_p
    L.pa_options_default.restype = None
    L.pa_options_default.argtypes = [C.POINTER(Options)]
    L.pa_create.restype = C.c_int
    L.pa_create.argtypes = [C.POINTER(vp), i32, i32, i64, vp, vp, vp, C.c_int,
                            C.POINTER(Options), vp]
    L.pa_estimate.restype = C.c_int
    L.pa_estimate.argtypes = [vp, C.c_int, C.c_int, d, d, d, d, u64, vp, vp, vp]
    L.pa_run.restype = C.c_int
    L.pa_run.argtypes = [vp, C.c_int, C.c_int, d, d, d, d, vp, C.c_int, vp, vp, vp, vp, vp,
                         C.c_int, vp]
    L.pa_estimate_batched.restype = C.c_int
    L.pa_estimate_batched.argtypes = [C.c_int, vp, C.c_int, C.c_int, vp, d, d, d, d, u64, vp, vp]
    L.pa_get_vector.restype = C.c_int
    L.pa_get_vector.argtypes = [vp, C.c_int, vp]
    L.pa_spmv.restype = C.c_int
    L.pa_spmv.argtypes = [vp, vp, vp, C.c_int]
    L.pa_spmv_t.restype = C.c_int
    L.pa_spmv_t.argtypes = [vp, vp, vp, C.c_int]
    L.pa_spmv_ata.restype = C.c_int
    L.pa_spmv_ata.argtypes = [vp, vp, vp, C.c_int]
    L.pa_launch_choice.restype = C.c_int
    L.pa_launch_choice.argtypes = [vp, vp, vp, vp]
    L.pa_single_pass_info.restype = C.c_int
    L.pa_single_pass_info.argtypes = [vp, vp]
    L.pa_lu_route_info.restype = C.c_int
    L.pa_lu_route_info.argtypes = [vp, vp]
    L.pa_get_transpose.restype = C.c_int
    L.pa_get_transpose.argtypes = [vp, vp, vp, vp]
    L.pa_get_equilibration.restype = C.c_int
    L.pa_get_equilibration.argtypes = [vp, vp, vp]
    L.pa_attach_lu.restype = C.c_int
    L.pa_attach_lu.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, C.c_int]
    L.pa_error_bounds.restype = C.c_int
    L.pa_error_bounds.argtypes = [vp, vp, vp, C.c_int, d, d, d, vp]
    L.pa_continue.restype = C.c_int
    L.pa_continue.argtypes = [vp, C.c_int, d, d, d, d, vp, vp, vp]
    L.pa_last_run_info.restype = C.c_int
    L.pa_last_run_info.argtypes = [vp, vp]
    L.pa_last_run_profile.restype = C.c_int
    L.pa_last_run_profile.argtypes = [vp, C.POINTER(C.c_int), vp]
    L.pa_last_batch_graph.restype = C.c_int
    L.pa_last_batch_graph.argtypes = []
    L.pa_sigma_noalloc.restype = C.c_int
    L.pa_sigma_noalloc.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp]
    L.pa_kernel_launches.restype = i64
    L.pa_kernel_launches.argtypes = [vp]
    L.pa_destroy.restype = None
    L.pa_destroy.argtypes = [vp]
    L.pa_last_error.restype = C.c_char_p
    L.pa_last_error.argtypes = []
    L.pa_set_allocator.restype = None
    L.pa_set_allocator.argtypes = [_ALLOC, _FREE, vp]


def _check(st: int, L=None) -> int:
    if st < 0:
        L = L or load()
        raise PAError(st, (L.pa_last_error() or b"").decode())
    return st


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _hooks
    import torch

    L = load()

    def _alloc(nbytes, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream(dev)
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, s)
        except Exception:  # noqa: BLE001 -- the library reports PA_ERR_OOM
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    _hooks = (_ALLOC(_alloc), _FREE(_free))
    L.pa_set_allocator(_hooks[0], _hooks[1], None)


def _ptr_and_kind(a, dtype):
    """(pointer, kind, keep-alive) for a numpy array (host) or torch CUDA tensor (device)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != dtype[1]:
                raise TypeError(f"expected {dtype[1]}, got {a.dtype}")
            if not a.is_contiguous():
                a = a.contiguous()
            return (a.data_ptr(), DEVICE if a.is_cuda else HOST, a)
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype[0])
    return (arr.ctypes.data, HOST, arr)


def _dtypes():
    try:
        import torch
        return {"i32": (np.int32, torch.int32), "f64": (np.float64, torch.float64)}
    except ImportError:
        return {"i32": (np.int32, None), "f64": (np.float64, None)}


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def options(**kw) -> Options:
    o = Options()
    load().pa_options_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Handle:
    """An A in CSR on the GPU (pa_create); see the C ABI for each method."""

    def __init__(self, raw, n_rows, n_cols, nnz, stream):
        self._h = raw
        self.n_rows, self.n_cols, self.nnz = n_rows, n_cols, nnz
        self.stream = stream

    @property
    def raw(self):
        return self._h

    def destroy(self):
        if self._h:
            load().pa_destroy(self._h)
            self._h = None

    close = destroy

    def __del__(self):
        try:
            self.destroy()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def launches(self) -> int:
        return int(load().pa_kernel_launches(self._h))

    def estimate(self, mode=BOTH, iters=2000, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12, seed=1):
        smax, smin, kap = C.c_double(), C.c_double(), C.c_double()
        st = _check(load().pa_estimate(self._h, mode, iters, lr, beta1, beta2, eps,
                                       seed & (2**64 - 1), C.byref(smax), C.byref(smin),
                                       C.byref(kap)))
        return {"status": st, "sigma_max": smax.value, "sigma_min": smin.value, "kappa": kap.value}

    def run(self, mode, iters, x_init, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12,
            trace_L=False, n_trace=0):
        n = self.n_cols
        xp, xk, keep = _ptr_and_kind(x_init, _dtypes()["f64"])
        x_min = np.empty(n)
        x_last = np.empty(n)
        info = np.empty(4)
        Lt = np.empty(max(iters, 1)) if trace_L else None
        Xt = np.empty((n_trace, n)) if n_trace > 0 else None
        sig = C.c_double()
        st = _check(load().pa_run(self._h, mode, iters, lr, beta1, beta2, eps, xp, xk,
                                  x_min.ctypes.data, x_last.ctypes.data, info.ctypes.data,
                                  None if Lt is None else Lt.ctypes.data,
                                  None if Xt is None else Xt.ctypes.data, n_trace,
                                  C.byref(sig)))
        del keep
        return {"status": st, "x_min": x_min, "x_last": x_last, "L_min": info[0],
                "t_min": int(info[1]), "L_last": info[2], "iters_run": int(info[3]),
                "L_trace": None if Lt is None else Lt[:iters], "x_trace": Xt, "sigma": sig.value}

    def get_vector(self, which):
        x = np.empty(self.n_cols)
        _check(load().pa_get_vector(self._h, which, x.ctypes.data))
        return x

    def _product(self, fn, vec, n_out):
        vp, kind, keep = _ptr_and_kind(vec, _dtypes()["f64"])
        if kind == DEVICE:
            import torch
            out = torch.empty(n_out, dtype=torch.float64, device=keep.device)
            _check(fn(self._h, vp, out.data_ptr(), DEVICE))
            return out
        out = np.empty(n_out)
        _check(fn(self._h, vp, out.ctypes.data, HOST))
        return out

    def spmv(self, x):
        return self._product(load().pa_spmv, x, self.n_rows)

    def spmv_t(self, y):
        return self._product(load().pa_spmv_t, y, self.n_cols)

    def spmv_ata(self, x):
        """pa_spmv_ata: A^T (A x) through the single-pass engine's plans."""
        return self._product(load().pa_spmv_ata, x, self.n_cols)

    def launch_choice(self):
        """pa_launch_choice: {kernel, grid, source, trials: [(kernel, grid, ms)]}."""
        out = np.zeros(4, dtype=np.int64)
        cand = np.zeros(8, dtype=np.int64)
        ms = np.zeros(4)
        _check(load().pa_launch_choice(self._h, out.ctypes.data, cand.ctypes.data, ms.ctypes.data))
        n = int(out[3])
        return dict(kernel=int(out[0]), grid=int(out[1]), source=int(out[2]),
                    trials=[(int(cand[2 * i]), int(cand[2 * i + 1]), float(ms[i])) for i in range(n)])

    def single_pass_info(self):
        """pa_single_pass_info: {grid, window_cols, plan_entries, plan_slots, groups,
        a_entries}."""
        out = np.zeros(6, dtype=np.int64)
        _check(load().pa_single_pass_info(self._h, out.ctypes.data))
        return dict(grid=int(out[0]), window_cols=int(out[1]), plan_entries=int(out[2]),
                    plan_slots=int(out[3]), groups=int(out[4]), a_entries=int(out[5]))

    def lu_route_info(self):
        """pa_lu_route_info: {route (0 one CTA, 1 grid, 2 cluster), ctas, cap, fin}."""
        out = np.zeros(4, dtype=np.int64)
        _check(load().pa_lu_route_info(self._h, out.ctypes.data))
        return dict(route=int(out[0]), ctas=int(out[1]), cap=int(out[2]), fin=int(out[3]))

    def get_transpose(self):
        rpt = np.empty(self.n_cols + 1, dtype=np.int32)
        cit = np.empty(max(self.nnz, 1), dtype=np.int32)
        vat = np.empty(max(self.nnz, 1))
        _check(load().pa_get_transpose(self._h, rpt.ctypes.data, cit.ctypes.data, vat.ctypes.data))
        return rpt, cit[:self.nnz], vat[:self.nnz]

    def last_run_profile(self):
        """(grid, busy_ns[grid, 2]) of the latest persistent run (phase A, phases B+C)."""
        g = C.c_int()
        _check(load().pa_last_run_profile(self._h, C.byref(g), None))
        t = np.zeros((max(g.value, 1), 2))
        _check(load().pa_last_run_profile(self._h, C.byref(g), t.ctypes.data))
        return g.value, t[:g.value]

    def continue_run(self, iters, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12):
        """pa_continue: the latest FP64 run continued for `iters` iterations;
        {status, sigma, x_last, L_min, t_min, L_last, iters_total}."""
        sig = C.c_double()
        x_last = np.empty(self.n_cols)
        info = np.empty(4)
        st = _check(load().pa_continue(self._h, int(iters), lr, beta1, beta2, eps, C.byref(sig),
                                       x_last.ctypes.data, info.ctypes.data))
        return {"status": st, "sigma": sig.value, "x_last": x_last, "L_min": info[0],
                "t_min": int(info[1]), "L_last": info[2], "iters_total": int(info[3])}

    def last_run_info(self):
        """pa_last_run_info: {kernel, refreshes, df_fallbacks, grid} of the
        latest single-vector run (kernel 0 three-phase grid, 1 merged FP64,
        2 merged double-float, 3 cluster, 4/5 LU route, 6 single-pass)."""
        out = np.zeros(4, dtype=np.int64)
        _check(load().pa_last_run_info(self._h, out.ctypes.data))
        return dict(kernel=int(out[0]), refreshes=int(out[1]), df_fallbacks=int(out[2]),
                    grid=int(out[3]))

    def attach_lu(self, L, U, p=None, q=None):
        """pa_attach_lu: P A Q = L U (L lower, U upper triangular, CSR given as
        synth.CSR / (row_ptr, col, val, n, n) on the host or as CUDA torch
        tensors); p[i] = row of A that is row i of P A, q[j] = column of A
        that is column j of A Q (None = identity)."""
        i32, f64 = _dtypes()["i32"], _dtypes()["f64"]
        keep = []

        def arrs(T):
            rp, ci, va = (T.row_ptr, T.col, T.val) if hasattr(T, "row_ptr") else T[:3]
            out = [_ptr_and_kind(rp, i32), _ptr_and_kind(ci, i32), _ptr_and_kind(va, f64)]
            keep.extend(out)
            return out

        Lp, Up = arrs(L), arrs(U)
        pp = _ptr_and_kind(p, i32) if p is not None else (None, None, None)
        qp = _ptr_and_kind(q, i32) if q is not None else (None, None, None)
        kinds = {a[1] for a in Lp + Up} | {k for k in (pp[1], qp[1]) if k is not None}
        if len(kinds) != 1:
            raise ValueError("factors and permutations must all be host arrays or all CUDA tensors")
        _check(load().pa_attach_lu(self._h, Lp[0][0], Lp[1][0], Lp[2][0], Up[0][0], Up[1][0],
                                   Up[2][0], pp[0], qp[0], kinds.pop()))

    def error_bounds(self, x_hat, b, kappa: float = 0.0, norm_a: float = 0.0,
                     u: float = 0.0) -> dict:
        """pa_error_bounds: residual of x_hat for A x = b and the bounds of the
        paper's Theorems 1-4 (kappa / norm_a <= 0: the handle's estimates)."""
        f64 = _dtypes()["f64"]
        xp, kx, keep_x = _ptr_and_kind(x_hat, f64)
        bp, kb, keep_b = _ptr_and_kind(b, f64)
        if kx != kb:
            raise ValueError("x_hat and b must both be host arrays or both device tensors")
        out = np.empty(10)
        _check(load().pa_error_bounds(self._h, xp, bp, kx, kappa, norm_a, u, out.ctypes.data))
        return dict(zip(ERROR_BOUND_KEYS, out.tolist()))

    def get_equilibration(self):
        dr, dc = np.empty(self.n_rows), np.empty(self.n_cols)
        _check(load().pa_get_equilibration(self._h, dr.ctypes.data, dc.ctypes.data))
        return dr, dc


def create(A, opts: Options | None = None, stream=None, **kw) -> Handle:
    """pa_create from a CSR given as ``synth.CSR`` / a tuple (row_ptr, col, val, n_rows, n_cols).

    numpy arrays are host pointers; CUDA torch tensors are device pointers.
    """
    row_ptr, col, val, n_rows, n_cols = A.astuple() if hasattr(A, "astuple") else A
    dt = _dtypes()
    rp, k1, keep1 = _ptr_and_kind(row_ptr, dt["i32"])
    ci, k2, keep2 = _ptr_and_kind(col, dt["i32"])
    va, k3, keep3 = _ptr_and_kind(val, dt["f64"])
    if len({k1, k2, k3}) != 1:
        raise ValueError("CSR arrays must all be host or all be device")
    nnz = int(keep2.shape[0]) if hasattr(keep2, "shape") else len(keep2)
    o = opts if opts is not None else options(**kw)
    raw = C.c_void_p()
    L = load()
    _check(L.pa_create(C.byref(raw), int(n_rows), int(n_cols), nnz, rp, ci, va, k1, C.byref(o),
                       _stream_ptr(stream)))
    del keep1, keep2, keep3
    return Handle(raw, int(n_rows), int(n_cols), nnz, stream)


def estimate_batched(handles, mode=BOTH, k_restarts=8, iters=(2000, 2000), lr=1e-2, beta1=0.9,
                     beta2=0.999, eps=1e-12, seed=1):
    n = len(handles)
    arr = (C.c_void_p * n)(*[h.raw for h in handles])
    it = (C.c_int * 2)(*iters)
    out = np.empty((n, k_restarts, 3))
    stat = np.empty((n, k_restarts), dtype=np.int32)
    st = _check(load().pa_estimate_batched(n, arr, mode, k_restarts, it, lr, beta1, beta2, eps,
                                           seed & (2**64 - 1), out.ctypes.data, stat.ctypes.data))
    return {"status": st, "sigma_max": out[:, :, 0], "sigma_min": out[:, :, 1],
            "kappa": out[:, :, 2], "item_status": stat,
            "cuda_graph": bool(load().pa_last_batch_graph())}


def sigma_noalloc(row_ptr, col, val, x, out, n_rows: int, n_cols: int, stream=None) -> int:
    """pa_sigma_noalloc: ||A x|| / ||x|| into out[0]; every argument is a CUDA
    torch tensor (row_ptr/col int32, val/x/out float64).  Enqueues only; the
    caller synchronises.  Returns the status (raises PAError on errors)."""
    return _check(load().pa_sigma_noalloc(int(n_rows), int(n_cols), row_ptr.data_ptr(),
                                          col.data_ptr(), val.data_ptr(), x.data_ptr(),
                                          out.data_ptr(), _stream_ptr(stream)))
