"""FP64 CPU oracle for IHT on PLINK-packed genotypes (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import this package.  The CUDA library never calls it and
shares no code with it.  ``iht_oracle.c`` holds the arithmetic; this module
only compiles it and marshals numpy arrays.

Parity pins (tests/test_oracle_*.py) tie every function here to something
other than itself: brute-force decoding, exact rational arithmetic, numpy's
nan-aware mean/std, least-squares closed forms, brute force over all k-subsets
and the invariants of the method.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iht_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, EINVAL, ENOMEM, ENOTCONV, ENUMERIC = 0, 1, 2, 3, 4


def build(force: bool = False, src: str = _SRC, out: str = _LIB, defines=()) -> str:
    """Compile the oracle (gcc -O2 -fopenmp, strict IEEE: no -ffast-math)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
               "-o", tmp, src, "-lm"] + [f"-D{d}" for d in defines]
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


class _Opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("max_backtrack", ctypes.c_int32),
                ("tol", ctypes.c_double), ("c", ctypes.c_double), ("kappa", ctypes.c_double),
                ("variant", ctypes.c_int32), ("pad", ctypes.c_int32)]


VARIANTS = {"iht": 0, "htp": 1}


class _Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("status", ctypes.c_int32),
                ("backtracks", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("objective", ctypes.c_double), ("mu", ctypes.c_double)]


class _Trace(ctypes.Structure):
    _fields_ = [(nm, ctypes.c_void_p) for nm in
                ("objective", "mu", "omega", "backtracks", "changed", "gap", "wscale",
                 "margin", "step", "supp", "beta")]


def load(path: str = _LIB, build_first: bool = True):
    """ctypes handle of an oracle build (the default build is cached)."""
    global _lib
    if path == _LIB and _lib is not None:
        return _lib
    if build_first and path == _LIB:
        build()
    lib = ctypes.CDLL(path)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.oracle_decode.argtypes = [P, i64, i64, i64, P]
    lib.oracle_counts.argtypes = [P, i64, i64, i64, P, i64, P, P, P]
    lib.oracle_gradient.argtypes = [P, i64, i64, i64, P, i64, P, P, P, P]
    lib.oracle_zmul.argtypes = [P, i64, i64, P, i64, P, P, P, i32, P, P]
    lib.oracle_topk.argtypes = [P, i64, i32, P]
    lib.oracle_iht.argtypes = [P, i64, i64, i64, P, i64, P, i32, ctypes.POINTER(_Opts), P, i64,
                               P, P, ctypes.POINTER(_Info), ctypes.POINTER(_Trace)]
    lib.oracle_cov_stats.argtypes = [P, i64, i64, P, i64, P, P]
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = None
    lib.oracle_max_threads.restype = ctypes.c_int
    for f in ("oracle_decode", "oracle_counts", "oracle_gradient", "oracle_zmul",
              "oracle_topk", "oracle_iht", "oracle_cov_stats"):
        getattr(lib, f).restype = ctypes.c_int
    if path == _LIB:
        _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data


def _rows(rows):
    return None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)


def _check(rc):
    if rc not in (OK, ENOTCONV):
        raise RuntimeError(f"oracle status {rc}")
    return rc


@dataclass
class Geno:
    """A .bed body (no header): p rows of ``row_bytes`` bytes, n subjects."""
    body: np.ndarray
    n: int
    p: int
    row_bytes: int

    @staticmethod
    def from_bed(bed: np.ndarray, n: int, p: int) -> "Geno":
        bed = np.ascontiguousarray(bed, dtype=np.uint8)
        if bed.size < 3 or bytes(bed[:3]) != bytes([0x6C, 0x1B, 0x01]):
            raise ValueError("not a SNP-major .bed image")
        rb = (n + 3) // 4
        if bed.size != 3 + p * rb:
            raise ValueError("size does not match n, p")
        return Geno(bed[3:], n, p, rb)


def set_threads(t: int, lib=None):
    (lib or load()).oracle_set_threads(int(t))


def max_threads(lib=None) -> int:
    return int((lib or load()).oracle_max_threads())


def decode(G: Geno, lib=None) -> np.ndarray:
    out = np.empty((G.p, G.n), dtype=np.int8)
    _check((lib or load()).oracle_decode(_p(G.body), G.row_bytes, G.n, G.p, _p(out)))
    return out


def counts(G: Geno, rows=None, lib=None):
    """(counts int32[p,4] by code, u float64[p], v float64[p])."""
    rows = _rows(rows)
    nr = G.n if rows is None else rows.size
    c = np.empty((G.p, 4), dtype=np.int32)
    u = np.empty(G.p)
    v = np.empty(G.p)
    _check((lib or load()).oracle_counts(_p(G.body), G.row_bytes, G.n, G.p, _p(rows), nr,
                                         _p(c), _p(u), _p(v)))
    return c, u, v


def gradient(G: Geno, r, rows=None, u=None, v=None, lib=None) -> np.ndarray:
    rows = _rows(rows)
    if u is None or v is None:
        _, u, v = counts(G, rows, lib)
    r = np.ascontiguousarray(r, dtype=np.float64)
    g = np.empty(G.p)
    _check((lib or load()).oracle_gradient(_p(G.body), G.row_bytes, G.n, G.p, _p(rows), r.size,
                                           _p(np.ascontiguousarray(u)), _p(np.ascontiguousarray(v)),
                                           _p(r), _p(g)))
    return g


def zmul(G: Geno, cols, coef, rows=None, u=None, v=None, lib=None) -> np.ndarray:
    """Z[rows, cols] @ coef with the given (or the rows') statistics."""
    rows = _rows(rows)
    if u is None or v is None:
        _, u, v = counts(G, rows, lib)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    nr = G.n if rows is None else rows.size
    out = np.empty(nr)
    _check((lib or load()).oracle_zmul(_p(G.body), G.row_bytes, G.n, _p(rows), nr,
                                       _p(np.ascontiguousarray(u)), _p(np.ascontiguousarray(v)),
                                       _p(cols), cols.size, _p(coef), _p(out)))
    return out


def _cov(cov, n: int):
    """Covariates as a contiguous (q, n) float64 array, or None."""
    if cov is None:
        return None
    c = np.ascontiguousarray(np.atleast_2d(cov), dtype=np.float64)
    if c.shape[1] != n:
        raise ValueError("cov must have shape (q, n)")
    return c


def cov_stats(cov, n: int, rows=None, lib=None):
    """Mean and inverse SD of each covariate over the rows (reading R13)."""
    c = _cov(cov, n)
    rows = _rows(rows)
    nr = n if rows is None else rows.size
    q = c.shape[0]
    cu, cv = np.empty(q), np.empty(q)
    _check((lib or load()).oracle_cov_stats(_p(c), n, q, _p(rows), nr, _p(cu), _p(cv)))
    return cu, cv


def topk(w, k: int, lib=None) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty(k, dtype=np.int32)
    _check((lib or load()).oracle_topk(_p(w), w.size, k, _p(out)))
    return out


@dataclass
class Fit:
    beta: np.ndarray
    support: np.ndarray
    iterations: int
    status: int
    backtracks: int
    objective: float
    mu: float
    trace: dict = field(default_factory=dict)


def iht(G: Geno, y, k: int, rows=None, max_iter: int = 100, tol: float = 1e-4, c: float = 0.01,
        kappa: float = 2.0, max_backtrack: int = 50, trace: bool = True, lib=None,
        variant: str = "iht", cov=None) -> Fit:
    """IHT (or HTP, variant="htp") on the SNPs and the optional covariates
    cov (q, n); beta has p + q entries, covariate t at index p + t."""
    rows = _rows(rows)
    y = np.ascontiguousarray(y, dtype=np.float64)
    cv = _cov(cov, G.n)
    q = 0 if cv is None else cv.shape[0]
    beta = np.zeros(G.p + q)
    supp = np.empty(k, dtype=np.int32)
    opts = _Opts(max_iter, max_backtrack, tol, c, kappa, VARIANTS[variant], 0)
    info = _Info()
    T = max(max_iter, 1)
    tr = {}
    ct = _Trace()
    if trace:
        tr = dict(objective=np.full(T, np.nan), mu=np.full(T, np.nan), omega=np.full(T, np.nan),
                  backtracks=np.zeros(T, np.int32), changed=np.zeros(T, np.int32),
                  gap=np.full(T, np.nan), wscale=np.full(T, np.nan), margin=np.full(T, np.nan),
                  step=np.full(T, np.nan), supp=np.zeros((T, k), np.int32),
                  beta=np.zeros((T, k)))
        for nm, arr in tr.items():
            setattr(ct, nm, arr.ctypes.data)
    rc = (lib or load()).oracle_iht(_p(G.body), G.row_bytes, G.n, G.p, _p(rows), y.size, _p(y),
                                    k, ctypes.byref(opts), _p(cv), q, _p(beta), _p(supp),
                                    ctypes.byref(info), ctypes.byref(ct) if trace else None)
    if rc not in (OK, ENOTCONV, ENUMERIC):
        raise RuntimeError(f"oracle_iht status {rc}")
    if trace:
        it = info.iterations
        tr = {nm: arr[:it] for nm, arr in tr.items()}
    return Fit(beta, supp, info.iterations, rc, info.backtracks, info.objective, info.mu, tr)


@dataclass
class CV:
    mse: np.ndarray          # [nk]: out-of-fold MSE averaged over the q folds
    mse_fold: np.ndarray     # [q, nk]: each fold's out-of-fold MSE
    k_best: int
    fit: Fit                 # the refit on all rows at k_best
    fits: list               # fits[f][t]: fold f's fit at ks[t]


def cv(G: Geno, y, fold, q: int, ks, max_iter: int = 100, tol: float = 1e-4, c: float = 0.01,
       kappa: float = 2.0, max_backtrack: int = 50, lib=None, trace: bool = False) -> CV:
    """q-fold cross-validation over the model sizes ks, then the refit (Sec. 2.4).

    fold[i] in 0..q-1 is subject i's partition, -1 a subject outside the
    selection and the refit (a held-out test set, as Sec. 3.1 keeps one apart
    from the cross-validation).  The path is fitted on the other
    q - 1 partitions (statistics of those rows); partition f is the test set:
    its MSE is the mean over its rows of (y_i - z_i^T beta)^2, z_i standardised
    with the training rows' statistics (the reading the batched solves use).
    The curve averages the q partitions' MSEs (the paper plots MSE averaged
    over the cross-validation slices); k_best is the first model size in ks
    with the least averaged MSE, and the model is refitted on all labelled rows
    with ||beta||_0 <= k_best.
    """
    y = np.ascontiguousarray(y, dtype=np.float64)
    fold = np.asarray(fold)
    ks = [int(k) for k in ks]
    kw = dict(max_iter=max_iter, tol=tol, c=c, kappa=kappa, max_backtrack=max_backtrack, lib=lib)
    mse_fold = np.zeros((q, len(ks)))
    fits = []
    for f in range(q):
        train = np.flatnonzero((fold != f) & (fold >= 0)).astype(np.int32)
        test = np.flatnonzero(fold == f).astype(np.int32)
        _, ut, vt = counts(G, train, lib)
        row = []
        for t, k in enumerate(ks):
            fit = iht(G, y[train], k, rows=train, trace=trace, **kw)
            pred = zmul(G, fit.support, fit.beta[fit.support], test, ut, vt, lib)
            mse_fold[f, t] = np.mean((y[test] - pred) ** 2)
            row.append(fit)
        fits.append(row)
    mse = mse_fold.mean(axis=0)
    k_best = ks[int(np.argmin(mse))]
    inside = np.flatnonzero(fold >= 0).astype(np.int32)
    refit = (iht(G, y, k_best, trace=trace, **kw) if inside.size == fold.size
             else iht(G, y[inside], k_best, rows=inside, trace=trace, **kw))
    return CV(mse, mse_fold, k_best, refit, fits)
