"""Python binding of libiht (include/iht.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does
nothing but check types, hand over pointers and turn status codes into
exceptions.  All work runs in the CUDA kernels of ``libiht.so``; there is no
CPU fallback, and loading fails loudly when the library or a CUDA device is
missing.  PyTorch supplies device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import mmap
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiht.so")

IHT_OK, IHT_EINVAL, IHT_ENOMEM, IHT_ENOTCONV, IHT_ENUMERIC, IHT_ETIMEOUT, IHT_ECUDA, IHT_EAGAIN = \
    range(8)
IHT_HOST, IHT_DEVICE = 0, 1
IHT_PASS_SINGLE, IHT_PASS_MULTI = 0, 1
IHT_FAULT_NONE, IHT_FAULT_ALLOC, IHT_FAULT_TIMEOUT = 0, 1, 2
IHT_VARIANT_IHT, IHT_VARIANT_HTP = 0, 1
IHT_FIT_BETA_ZEROED = 1
VARIANTS = {"iht": IHT_VARIANT_IHT, "htp": IHT_VARIANT_HTP}

EXPORTED = ["iht_default_options", "iht_strerror", "iht_last_cuda_error", "iht_kernel_launches",
            "iht_create",
            "iht_destroy", "iht_load_bed", "iht_dataset_free", "iht_dataset_shape", "iht_counts",
            "iht_gradient", "iht_topk", "iht_topk_noalloc", "iht_zmul", "iht_fit",
            "iht_fit_trace", "iht_fit_batch", "iht_gradient_batch", "iht_server_default_options",
            "iht_server_create", "iht_server_submit", "iht_server_poll", "iht_server_get_stats",
            "iht_server_destroy", "iht_state_bytes", "iht_state_save", "iht_state_load",
            "iht_fit_resume", "iht_set_autotune", "iht_tune_clear", "iht_tune_pin", "iht_tune_query",
            "iht_tuning_summary", "iht_cv", "iht_fault_inject", "iht_set_covariates"]


class IhtError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = f"{where}: {status_name(status)}"
        if status == IHT_ECUDA:
            msg += f" [{_lib().iht_last_cuda_error().decode()}]"
        super().__init__(msg)
        self.status = status


class iht_options(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("max_backtrack", ctypes.c_int32),
                ("tol", ctypes.c_double), ("c", ctypes.c_double), ("kappa", ctypes.c_double),
                ("in_mem", ctypes.c_int32), ("out_mem", ctypes.c_int32),
                ("grad_impl", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("flags", ctypes.c_int32)]


class iht_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("status", ctypes.c_int32),
                ("backtracks", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("objective", ctypes.c_double), ("mu", ctypes.c_double),
                ("grad_ms", ctypes.c_double), ("grad_launches", ctypes.c_int32),
                ("graph_replays", ctypes.c_int32)]


class iht_trace(ctypes.Structure):
    _fields_ = [("objective", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("backtracks", ctypes.c_void_p), ("changed", ctypes.c_void_p),
                ("supp", ctypes.c_void_p), ("beta", ctypes.c_void_p)]


class iht_solve_desc(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_void_p), ("n_rows", ctypes.c_int64), ("y", ctypes.c_void_p),
                ("k", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class iht_server_options(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("hbm_budget", ctypes.c_uint64), ("solve", iht_options)]


class iht_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("ticks", ctypes.c_uint64),
                ("active", ctypes.c_int32), ("max_active", ctypes.c_int32),
                ("bytes_in_use", ctypes.c_uint64), ("max_bytes_in_use", ctypes.c_uint64)]


_LIB = None


def _lib(build_if_stale: bool = True):
    """The loaded libiht.so (compiled in-tree when missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_stale:
        from . import build as _build
        try:
            if _build.stale():
                _build.build()
        except (OSError, RuntimeError) as e:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libiht.so is missing and could not be built: {e}") from e
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libiht.so not found at {LIB_PATH}")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "iht_default_options": (None, [ctypes.POINTER(iht_options)]),
        "iht_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "iht_last_cuda_error": (ctypes.c_char_p, []),
        "iht_kernel_launches": (ctypes.c_uint64, []),
        "iht_fault_inject": (ctypes.c_int, [ctypes.c_int, i32]),
        "iht_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, P]),
        "iht_destroy": (ctypes.c_int, [P]),
        "iht_load_bed": (ctypes.c_int, [P, P, sz, ctypes.c_int, i64, i64, ctypes.POINTER(P)]),
        "iht_dataset_free": (ctypes.c_int, [P]),
        "iht_set_covariates": (ctypes.c_int, [P, P, i32, ctypes.c_int]),
        "iht_dataset_shape": (ctypes.c_int, [P, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                             ctypes.POINTER(i64)]),
        "iht_counts": (ctypes.c_int, [P, P, i64, ctypes.c_int, P, P, P]),
        "iht_gradient": (ctypes.c_int, [P, P, i64, P, P, ctypes.c_int]),
        "iht_topk": (ctypes.c_int, [P, P, i64, i32, P]),
        "iht_topk_noalloc": (ctypes.c_int, [ctypes.c_int, P, P, i64, i32, P]),
        "iht_zmul": (ctypes.c_int, [P, P, i64, P, P, P, i32, P, P]),
        "iht_fit": (ctypes.c_int, [P, P, i64, P, i32, ctypes.POINTER(iht_options), P, P,
                                   ctypes.POINTER(iht_result)]),
        "iht_fit_trace": (ctypes.c_int, [P, P, i64, P, i32, ctypes.POINTER(iht_options), P, P,
                                         ctypes.POINTER(iht_result), ctypes.POINTER(iht_trace)]),
        "iht_fit_batch": (ctypes.c_int, [P, i32, ctypes.POINTER(iht_solve_desc),
                                         ctypes.POINTER(iht_options), P, P, P,
                                         ctypes.POINTER(iht_result)]),
        "iht_gradient_batch": (ctypes.c_int, [P, i32, ctypes.POINTER(P), ctypes.POINTER(i64), P, P,
                                              ctypes.c_int]),
        "iht_server_default_options": (None, [ctypes.POINTER(iht_server_options)]),
        "iht_server_create": (ctypes.c_int, [P, ctypes.POINTER(iht_server_options),
                                             ctypes.POINTER(P)]),
        "iht_server_submit": (ctypes.c_int, [P, ctypes.POINTER(iht_solve_desc),
                                             ctypes.POINTER(ctypes.c_uint64)]),
        "iht_server_poll": (ctypes.c_int, [P, ctypes.c_uint64, P, P, ctypes.POINTER(iht_result),
                                           ctypes.POINTER(ctypes.c_double)]),
        "iht_server_get_stats": (ctypes.c_int, [P, ctypes.POINTER(iht_server_stats)]),
        "iht_server_destroy": (ctypes.c_int, [P]),
        "iht_state_bytes": (ctypes.c_int, [i32, ctypes.POINTER(sz)]),
        "iht_state_save": (ctypes.c_int, [i64, i64, i64, i32, P, P, ctypes.POINTER(iht_result), P,
                                          sz]),
        "iht_state_load": (ctypes.c_int, [P, sz, i32, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                          ctypes.POINTER(i64), ctypes.POINTER(i32), P, P,
                                          ctypes.POINTER(iht_result)]),
        "iht_fit_resume": (ctypes.c_int, [P, P, i64, P, P, sz, ctypes.POINTER(iht_options), P, P,
                                          ctypes.POINTER(iht_result)]),
        "iht_set_autotune": (None, [ctypes.c_int]),
        "iht_tune_clear": (None, []),
        "iht_tune_pin": (ctypes.c_int, [P, i32, i32, P, i32]),
        "iht_tune_query": (ctypes.c_int, [P, i32, i32, P, i32]),
        "iht_tuning_summary": (ctypes.c_int, [P, sz]),
        "iht_cv": (ctypes.c_int, [P, P, P, i32, P, i32, ctypes.POINTER(iht_options), P, P,
                                  ctypes.POINTER(i32), P, P, ctypes.POINTER(iht_result)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def iht_kernel_launches() -> int:
    """Kernel launches issued by libiht in this process."""
    return int(_lib().iht_kernel_launches())


def fault_inject(kind: int, count: int = 1) -> None:
    """Host-side fault injection for error-path tests (iht_fault_inject)."""
    _check(_lib().iht_fault_inject(int(kind), int(count)), "iht_fault_inject")


def status_name(s: int) -> str:
    return _lib().iht_strerror(int(s)).decode()


def _check(rc: int, where: str, ok=(IHT_OK,)):
    if rc not in ok:
        raise IhtError(rc, where)
    return rc


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libiht needs a CUDA device; none is visible")
    return torch


def _dptr(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    return t.data_ptr()


class Context:
    """iht_create / iht_destroy.  Orders work on the given torch stream."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        _check(_lib().iht_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream)),
               "iht_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib().iht_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Dataset:
    """iht_load_bed / iht_dataset_free."""

    def __init__(self, ctx: Context, bed, n: int, p: int):
        torch = _torch()
        self.ctx = ctx
        h = ctypes.c_void_p()
        if isinstance(bed, torch.Tensor):
            ptr, nbytes, mem = _dptr(bed, torch.uint8, "bed"), bed.numel(), IHT_DEVICE
        else:
            bed = np.ascontiguousarray(bed, dtype=np.uint8)
            ptr, nbytes, mem = bed.ctypes.data, bed.size, IHT_HOST
        _check(_lib().iht_load_bed(ctx.h, ctypes.c_void_p(ptr), nbytes, mem, n, p,
                                   ctypes.byref(h)), "iht_load_bed")
        self.h = h
        n_, p_, s_ = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _lib().iht_dataset_shape(h, ctypes.byref(n_), ctypes.byref(p_), ctypes.byref(s_))
        self.n, self.p, self.stride = n_.value, p_.value, s_.value
        self.q = 0

    def set_covariates(self, cov) -> None:
        """iht_set_covariates: cov (q, n) host array or CUDA float64 tensor; None
        or q = 0 removes them.  Fits then have p + q coefficients."""
        torch = _torch()
        if cov is None:
            _check(_lib().iht_set_covariates(self.h, None, 0, IHT_HOST), "iht_set_covariates")
            self.q = 0
            return
        if isinstance(cov, torch.Tensor):
            if cov.dim() != 2 or cov.shape[1] != self.n:
                raise ValueError("cov must have shape (q, n)")
            ptr, q, mem = _dptr(cov, torch.float64, "cov"), cov.shape[0], IHT_DEVICE
        else:
            cov = np.ascontiguousarray(np.atleast_2d(cov), dtype=np.float64)
            if cov.shape[1] != self.n:
                raise ValueError("cov must have shape (q, n)")
            ptr, q, mem = cov.ctypes.data, cov.shape[0], IHT_HOST
        _check(_lib().iht_set_covariates(self.h, ctypes.c_void_p(ptr), q, mem), "iht_set_covariates")
        self.q = q

    def close(self):
        if getattr(self, "h", None):
            _lib().iht_dataset_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def iht_default_options(**kw) -> iht_options:
    o = iht_options()
    _lib().iht_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        if k == "variant" and isinstance(v, str):
            v = VARIANTS[v]
        setattr(o, k, v)
    return o


def iht_counts(ds: Dataset, rows=None):
    """Host call: (counts int32[p,4], u float64[p], v float64[p])."""
    c = np.empty((ds.p, 4), dtype=np.int32)
    u = np.empty(ds.p)
    v = np.empty(ds.p)
    if rows is not None:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
    _check(_lib().iht_counts(ds.h, None if rows is None else ctypes.c_void_p(rows.ctypes.data),
                             0 if rows is None else rows.size, IHT_HOST,
                             ctypes.c_void_p(c.ctypes.data), ctypes.c_void_p(u.ctypes.data),
                             ctypes.c_void_p(v.ctypes.data)), "iht_counts")
    return c, u, v


def iht_gradient(ds: Dataset, r, rows=None, impl: int = 0, out=None):
    """g = Z^T r on the device; r float32 CUDA tensor aligned with rows."""
    torch = _torch()
    g = out if out is not None else torch.empty(ds.p, dtype=torch.float32, device=r.device)
    rp = None if rows is None else ctypes.c_void_p(_dptr(rows, torch.int32, "rows"))
    nr = ds.n if rows is None else rows.numel()
    if r.numel() != nr:
        raise ValueError("r must have one entry per row")
    _check(_lib().iht_gradient(ds.h, rp, nr, ctypes.c_void_p(_dptr(r, torch.float32, "r")),
                               ctypes.c_void_p(_dptr(g, torch.float32, "g")), impl), "iht_gradient")
    return g


def iht_topk(ctx: Context, w, k: int, out=None):
    """Indices of the k largest |w| (ties to the lower index), ascending."""
    torch = _torch()
    idx = out if out is not None else torch.empty(k, dtype=torch.int32, device=w.device)
    _check(_lib().iht_topk(ctx.h, ctypes.c_void_p(_dptr(w, torch.float32, "w")), w.numel(), k,
                           ctypes.c_void_p(_dptr(idx, torch.int32, "idx"))), "iht_topk")
    return idx


def iht_topk_noalloc(w, k: int, out, device: int | None = None, stream=None):
    """Allocation-free top-k: enqueues on `stream` (default: torch's current
    stream of w's device) and writes the k indices into `out` (int32, k).
    Marshalling only; the caller owns `out` and synchronises."""
    torch = _torch()
    dev = w.device.index if device is None else device
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    _check(_lib().iht_topk_noalloc(dev, ctypes.c_void_p(st.cuda_stream),
                                   ctypes.c_void_p(_dptr(w, torch.float32, "w")), w.numel(), k,
                                   ctypes.c_void_p(_dptr(out, torch.int32, "out"))),
           "iht_topk_noalloc")
    return out


def iht_zmul(ds: Dataset, cols, coef, rows=None, u=None, v=None):
    """Z[rows, cols] @ coef (FP64) on the device."""
    torch = _torch()
    nr = ds.n if rows is None else rows.numel()
    out = torch.empty(nr, dtype=torch.float64, device=coef.device)
    rp = None if rows is None else ctypes.c_void_p(_dptr(rows, torch.int32, "rows"))
    up = None if u is None else ctypes.c_void_p(_dptr(u, torch.float64, "u"))
    vp = None if v is None else ctypes.c_void_p(_dptr(v, torch.float64, "v"))
    _check(_lib().iht_zmul(ds.h, rp, nr, up, vp, ctypes.c_void_p(_dptr(cols, torch.int32, "cols")),
                           cols.numel(), ctypes.c_void_p(_dptr(coef, torch.float64, "coef")),
                           ctypes.c_void_p(out.data_ptr())), "iht_zmul")
    return out


@dataclass
class FitResult:
    beta: object
    support: object
    iterations: int
    status: int
    backtracks: int
    objective: float
    mu: float
    trace: dict | None = None
    grad_ms: float = 0.0
    grad_launches: int = 0
    beta_s: object = None
    graph_replays: int = 0


def _zeroed_f64(n: int) -> np.ndarray:
    """n zero doubles.  Large ones come from an anonymous mapping: its pages
    are zero until written, so a mostly-zero result (a k-sparse beta) costs a
    page fault per written page instead of clearing the whole array (a heap
    allocation that calloc must clear)."""
    if n * 8 < (1 << 20):
        return np.zeros(n)
    return np.frombuffer(mmap.mmap(-1, n * 8), dtype=np.float64)


def _fit(ds: Dataset, y, k: int, rows, opts: iht_options, trace: bool, state: bytes = None):
    torch = _torch()
    dev_in = isinstance(y, torch.Tensor)
    if dev_in:
        yp = _dptr(y, torch.float64, "y")
        nr = y.numel()
        rp = None if rows is None else _dptr(rows, torch.int32, "rows")
        opts.in_mem = IHT_DEVICE
    else:
        y = np.ascontiguousarray(y, dtype=np.float64)
        yp, nr = y.ctypes.data, y.size
        if rows is not None:
            rows = np.ascontiguousarray(rows, dtype=np.int32)
        rp = None if rows is None else rows.ctypes.data
        opts.in_mem = IHT_HOST
    if rows is None and nr != ds.n:
        raise ValueError("y must have n entries when rows is None")
    P = ds.p + ds.q                       # SNPs, then covariates
    if opts.out_mem == IHT_DEVICE:
        beta = torch.empty(P, dtype=torch.float64, device=f"cuda:{ds.ctx.device}")
        supp = torch.empty(k, dtype=torch.int32, device=f"cuda:{ds.ctx.device}")
        bp, sp = beta.data_ptr(), supp.data_ptr()
    else:
        beta = _zeroed_f64(P)             # zero pages: the library writes the support only
        opts.flags |= IHT_FIT_BETA_ZEROED
        supp = np.empty(k, dtype=np.int32)
        bp, sp = beta.ctypes.data, supp.ctypes.data
    res = iht_result()
    tr = None
    if state is not None:
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        rc = _lib().iht_fit_resume(ds.h, None if rp is None else ctypes.c_void_p(rp), nr,
                                   ctypes.c_void_p(yp), buf, len(state), ctypes.byref(opts),
                                   ctypes.c_void_p(bp), ctypes.c_void_p(sp), ctypes.byref(res))
    elif trace:
        T = max(opts.max_iter, 1)
        tr = dict(objective=np.full(T, np.nan), mu=np.full(T, np.nan),
                  backtracks=np.zeros(T, np.int32), changed=np.zeros(T, np.int32),
                  supp=np.zeros((T, k), np.int32), beta=np.zeros((T, k)))
        ct = iht_trace(*(tr[f].ctypes.data for f in
                         ("objective", "mu", "backtracks", "changed", "supp", "beta")))
        rc = _lib().iht_fit_trace(ds.h, None if rp is None else ctypes.c_void_p(rp), nr,
                                  ctypes.c_void_p(yp), k, ctypes.byref(opts), ctypes.c_void_p(bp),
                                  ctypes.c_void_p(sp), ctypes.byref(res), ctypes.byref(ct))
    else:
        rc = _lib().iht_fit(ds.h, None if rp is None else ctypes.c_void_p(rp), nr,
                            ctypes.c_void_p(yp), k, ctypes.byref(opts), ctypes.c_void_p(bp),
                            ctypes.c_void_p(sp), ctypes.byref(res))
    _check(rc, "iht_fit", ok=(IHT_OK, IHT_ENOTCONV, IHT_ENUMERIC))
    if tr is not None:
        tr = {f: a[:res.iterations] for f, a in tr.items()}
    return FitResult(beta, supp, res.iterations, rc, res.backtracks, res.objective, res.mu, tr,
                     res.grad_ms, res.grad_launches, None, res.graph_replays)


def iht_fit(ds: Dataset, y, k: int, rows=None, **opt) -> FitResult:
    """IHT to convergence.  y (and rows) numpy -> host inputs, CUDA tensors -> device inputs."""
    out_device = opt.pop("out_device", False)
    o = iht_default_options(**opt)
    o.out_mem = IHT_DEVICE if out_device else IHT_HOST
    return _fit(ds, y, k, rows, o, trace=False)


@dataclass
class SolveState:
    """A parsed solve-state image (see save_state / iht_fit_resume)."""
    n: int
    p: int
    n_rows: int
    k: int
    support: np.ndarray
    beta_s: np.ndarray
    iterations: int
    backtracks: int
    status: int
    objective: float
    mu: float


def save_state(shape, n_rows: int, fit: FitResult) -> bytes:
    """Checkpoint image of a stopped solve (iht_state_save; no device work).

    shape: (n, p) of the dataset (or the Dataset); n_rows: rows the solve used.
    """
    n, p = (shape.n, shape.p) if isinstance(shape, Dataset) else shape

    def host(a):                                   # device tensors come back; no device needed
        return a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)

    supp = np.ascontiguousarray(host(fit.support), dtype=np.int32)
    bs = host(fit.beta_s) if fit.beta_s is not None else host(fit.beta)[supp]
    bs = np.ascontiguousarray(bs, dtype=np.float64)
    k = supp.size
    nbytes = ctypes.c_size_t()
    _check(_lib().iht_state_bytes(k, ctypes.byref(nbytes)), "iht_state_bytes")
    info = iht_result(iterations=fit.iterations, status=fit.status, backtracks=fit.backtracks,
                      objective=fit.objective, mu=fit.mu)
    buf = ctypes.create_string_buffer(nbytes.value)
    _check(_lib().iht_state_save(n, p, n_rows, k, supp.ctypes.data, bs.ctypes.data,
                                 ctypes.byref(info), buf, nbytes.value), "iht_state_save")
    return buf.raw


def load_state(image: bytes) -> SolveState:
    """Parse a solve-state image (iht_state_load; raises IhtError when it is malformed)."""
    L = _lib()
    buf = ctypes.create_string_buffer(bytes(image), len(image))
    n, p, nr, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(L.iht_state_load(buf, len(image), 0, ctypes.byref(n), ctypes.byref(p), ctypes.byref(nr),
                            ctypes.byref(k), None, None, None), "iht_state_load")
    supp = np.empty(k.value, np.int32)
    bs = np.empty(k.value)
    info = iht_result()
    _check(L.iht_state_load(buf, len(image), k.value, ctypes.byref(n), ctypes.byref(p),
                            ctypes.byref(nr), ctypes.byref(k), supp.ctypes.data, bs.ctypes.data,
                            ctypes.byref(info)), "iht_state_load")
    return SolveState(n.value, p.value, nr.value, k.value, supp, bs, info.iterations,
                      info.backtracks, info.status, info.objective, info.mu)


def iht_fit_resume(ds: Dataset, y, state: bytes, rows=None, **opt) -> FitResult:
    """iht_fit continued from a checkpoint image; max_iter caps the total iterations."""
    out_device = opt.pop("out_device", False)
    o = iht_default_options(**opt)
    o.out_mem = IHT_DEVICE if out_device else IHT_HOST
    return _fit(ds, y, load_state(state).k, rows, o, trace=False, state=state)


@dataclass
class CVResult:
    mse: np.ndarray          # [nk] out-of-fold MSE averaged over the partitions
    mse_fold: np.ndarray     # [q, nk]
    k_best: int
    fit: FitResult           # refit on all rows at k_best


def iht_cv(ds: Dataset, y, fold, ks, q: int = None, **opt) -> CVResult:
    """q-fold cross-validation over the model sizes ks and the refit (iht_cv).

    y: host phenotype (n); fold: host partition label per subject (0..q-1, or
    -1 for a subject left out of the selection and the refit).
    """
    y = np.ascontiguousarray(y, dtype=np.float64)
    fold = np.ascontiguousarray(fold, dtype=np.int32)
    ks = np.ascontiguousarray(ks, dtype=np.int32)
    q = int(fold.max()) + 1 if q is None else int(q)
    o = iht_default_options(**opt)
    mse = np.empty(ks.size)
    mse_fold = np.empty((q, ks.size))
    kb = ctypes.c_int32()
    beta = np.empty(ds.p)
    supp = np.empty(int(ks.max()), np.int32)
    info = iht_result()
    rc = _lib().iht_cv(ds.h, y.ctypes.data, fold.ctypes.data, q, ks.ctypes.data, ks.size,
                       ctypes.byref(o), mse.ctypes.data, mse_fold.ctypes.data, ctypes.byref(kb),
                       beta.ctypes.data, supp.ctypes.data, ctypes.byref(info))
    _check(rc, "iht_cv", ok=(IHT_OK, IHT_ENOTCONV))
    k = kb.value
    fit = FitResult(beta, supp[:k].copy(), info.iterations, rc, info.backtracks, info.objective,
                    info.mu, None, info.grad_ms, info.grad_launches, beta[supp[:k]].copy(),
                    info.graph_replays)
    return CVResult(mse, mse_fold, k, fit)


def set_autotune(on: bool) -> None:
    """Turn the gradient passes' shape tuning on or off (iht_set_autotune)."""
    _lib().iht_set_autotune(1 if on else 0)


def tune_clear() -> None:
    """Forget every cached pass shape (iht_tune_clear)."""
    _lib().iht_tune_clear()


def _nparams(kind: int) -> int:
    return 1 if kind == IHT_PASS_SINGLE else 5


def tune_pin(ds: Dataset, kind: int, ncols: int, params) -> None:
    """Pin the launch shape of passes of `kind` over ncols columns (iht_tune_pin)."""
    a = np.ascontiguousarray(params, dtype=np.int32)
    _check(_lib().iht_tune_pin(ds.h, kind, ncols, a.ctypes.data, a.size), "iht_tune_pin")


def tune_query(ds: Dataset, kind: int, ncols: int):
    """Cached shape of passes of `kind` over ncols columns as a tuple, or None."""
    a = np.zeros(_nparams(kind), np.int32)
    rc = _lib().iht_tune_query(ds.h, kind, ncols, a.ctypes.data, a.size)
    if rc == IHT_EAGAIN:
        return None
    _check(rc, "iht_tune_query")
    return tuple(int(v) for v in a)


def tuning_summary() -> str:
    """The tuned / pinned shapes of this process, one line each (iht_tuning_summary)."""
    L = _lib()
    need = L.iht_tuning_summary(None, 0)
    buf = ctypes.create_string_buffer(max(need, 1))
    _check(L.iht_tuning_summary(buf, len(buf)), "iht_tuning_summary")
    return buf.value.decode()


def iht_fit_trace(ds: Dataset, y, k: int, rows=None, **opt) -> FitResult:
    out_device = opt.pop("out_device", False)
    o = iht_default_options(**opt)
    o.out_mem = IHT_DEVICE if out_device else IHT_HOST
    return _fit(ds, y, k, rows, o, trace=True)


def iht_fit_batch(ds: Dataset, problems, out_device: bool = False, dense: bool = True,
                  **opt) -> list:
    """b solves sharing the genotype passes (iht_fit_batch).

    problems: sequence of (y, k, rows); y and rows numpy arrays (host inputs)
    or CUDA tensors (device inputs), all of the same kind; rows None = all n.
    The same rows object in several problems is one row set (statistics
    computed once).  Returns one FitResult per problem with the support, beta
    on it (beta_s) and, when dense, the full coefficient vector (beta).
    """
    torch = _torch()
    o = iht_default_options(**opt)
    o.out_mem = IHT_DEVICE if out_device else IHT_HOST
    b = len(problems)
    if b < 1:
        raise ValueError("no problems")
    dev_in = isinstance(problems[0][0], torch.Tensor)
    o.in_mem = IHT_DEVICE if dev_in else IHT_HOST
    keep, rows_ptr = [], {}
    descs = (iht_solve_desc * b)()
    ks = []
    for c, (y, k, rows) in enumerate(problems):
        if isinstance(y, torch.Tensor) != dev_in:
            raise TypeError("all phenotypes must be host arrays or all CUDA tensors")
        if dev_in:
            yp, nr = _dptr(y, torch.float64, "y"), y.numel()
        else:
            y = np.ascontiguousarray(y, dtype=np.float64)
            yp, nr = y.ctypes.data, y.size
        keep.append(y)
        rp = None
        if rows is not None:
            key = id(rows)
            if key not in rows_ptr:
                if dev_in:
                    rows_ptr[key] = (_dptr(rows, torch.int32, "rows"), rows.numel(), rows)
                else:
                    ra = np.ascontiguousarray(rows, dtype=np.int32)
                    rows_ptr[key] = (ra.ctypes.data, ra.size, ra)
            rp, nrr, _ = rows_ptr[key]
            if nrr != nr:
                raise ValueError("y must have one entry per row")
        elif nr != ds.n:
            raise ValueError("y must have n entries when rows is None")
        descs[c] = iht_solve_desc(rp, nr, yp, int(k), 0)
        ks.append(int(k))
    ktot = sum(ks)
    if out_device:
        dev = f"cuda:{ds.ctx.device}"
        betas = torch.empty((b, ds.p), dtype=torch.float64, device=dev) if dense else None
        supp = torch.empty(ktot, dtype=torch.int32, device=dev)
        bsv = torch.empty(ktot, dtype=torch.float64, device=dev)
        bp = None if betas is None else betas.data_ptr()
        sp, vp = supp.data_ptr(), bsv.data_ptr()
    else:
        betas = np.empty((b, ds.p)) if dense else None
        supp = np.empty(ktot, dtype=np.int32)
        bsv = np.empty(ktot)
        bp = None if betas is None else betas.ctypes.data
        sp, vp = supp.ctypes.data, bsv.ctypes.data
    infos = (iht_result * b)()
    rc = _lib().iht_fit_batch(ds.h, b, descs, ctypes.byref(o), ctypes.c_void_p(bp),
                              ctypes.c_void_p(sp), ctypes.c_void_p(vp), infos)
    _check(rc, "iht_fit_batch")
    out, off = [], 0
    for c in range(b):
        r = infos[c]
        out.append(FitResult(None if betas is None else betas[c], supp[off:off + ks[c]],
                             r.iterations, r.status, r.backtracks, r.objective, r.mu, None,
                             r.grad_ms, r.grad_launches, bsv[off:off + ks[c]], r.graph_replays))
        off += ks[c]
    return out


def iht_gradient_batch(ds: Dataset, R, rows_list=None, impl: int = 0):
    """G[c] = Z_c^T r_c for b residual columns (float32 CUDA tensors, each
    aligned with its rows; rows_list entries None = all n).  Returns a (b, p)
    float32 CUDA tensor."""
    torch = _torch()
    b = len(R)
    rows_list = [None] * b if rows_list is None else list(rows_list)
    if len(rows_list) != b or b < 1:
        raise ValueError("one row list per column")
    dev = f"cuda:{ds.ctx.device}"
    Rbuf = torch.zeros((b, ds.n), dtype=torch.float32, device=dev)
    ptrs = (ctypes.c_void_p * b)()
    nrows = (ctypes.c_int64 * b)()
    for c in range(b):
        r, rows = R[c], rows_list[c]
        nr = ds.n if rows is None else rows.numel()
        if r.numel() != nr:
            raise ValueError("each column needs one entry per row")
        _dptr(r, torch.float32, "R[c]")
        Rbuf[c, :nr] = r
        ptrs[c] = None if rows is None else _dptr(rows, torch.int32, "rows")
        nrows[c] = nr
    G = torch.empty((b, ds.p), dtype=torch.float32, device=dev)
    _check(_lib().iht_gradient_batch(ds.h, b, ptrs, nrows, ctypes.c_void_p(Rbuf.data_ptr()),
                                     ctypes.c_void_p(G.data_ptr()), impl), "iht_gradient_batch")
    return G


@dataclass
class ServedResult:
    support: np.ndarray
    beta_s: np.ndarray
    iterations: int
    status: int
    backtracks: int
    objective: float
    mu: float
    latency_s: float


class Server:
    """iht_server_*: continuous-batching IHT solves on one dataset.

    submit() queues a request (host y and rows, copied) and returns a ticket;
    poll() returns None while it is queued or running, then its ServedResult
    (once).  The server's worker runs on its own stream of the dataset's
    device until close()."""

    def __init__(self, ds: Dataset, max_slots: int = 64, hbm_budget: int = 0, **solve):
        _torch()
        o = iht_server_options()
        _lib().iht_server_default_options(ctypes.byref(o))
        o.max_slots = max_slots
        o.hbm_budget = hbm_budget
        for k, v in solve.items():
            if not hasattr(o.solve, k):
                raise AttributeError(k)
            setattr(o.solve, k, v)
        h = ctypes.c_void_p()
        _check(_lib().iht_server_create(ds.h, ctypes.byref(o), ctypes.byref(h)), "iht_server_create")
        self.h = h
        self.ds = ds
        self._k = {}

    def submit(self, y, k: int, rows=None) -> int:
        y = np.ascontiguousarray(y, dtype=np.float64)
        if rows is not None:
            rows = np.ascontiguousarray(rows, dtype=np.int32)
            if rows.size != y.size:
                raise ValueError("y must have one entry per row")
        elif y.size != self.ds.n:
            raise ValueError("y must have n entries when rows is None")
        d = iht_solve_desc(None if rows is None else rows.ctypes.data, y.size, y.ctypes.data, int(k), 0)
        t = ctypes.c_uint64()
        _check(_lib().iht_server_submit(self.h, ctypes.byref(d), ctypes.byref(t)), "iht_server_submit")
        self._k[t.value] = int(k)
        return t.value

    def poll(self, ticket: int):
        k = self._k[ticket]
        supp = np.empty(k, dtype=np.int32)
        bs = np.empty(k)
        info = iht_result()
        lat = ctypes.c_double()
        rc = _lib().iht_server_poll(self.h, ticket, ctypes.c_void_p(supp.ctypes.data),
                                    ctypes.c_void_p(bs.ctypes.data), ctypes.byref(info),
                                    ctypes.byref(lat))
        if rc == IHT_EAGAIN:
            return None
        _check(rc, "iht_server_poll")
        del self._k[ticket]
        return ServedResult(supp, bs, info.iterations, info.status, info.backtracks, info.objective,
                            info.mu, lat.value)

    def stats(self) -> dict:
        st = iht_server_stats()
        _check(_lib().iht_server_get_stats(self.h, ctypes.byref(st)), "iht_server_get_stats")
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if getattr(self, "h", None):
            _lib().iht_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
