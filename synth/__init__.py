"""Seeded synthetic GWAS inputs, shared by the oracle tests, the GPU tests and the bench.

Nothing here computes any step of the method: the module draws allele
frequencies, genotype codes (through ``synth.c``), causal effects, noise and
row subsets, and writes genotypes in the PLINK ``.bed`` byte layout.  The
phenotype recipe standardises with the *population* allele frequency q_j
(z = (x - 2q)/sqrt(2q(1-q)), missing -> 0), never with the sample statistics
the method computes, so no value here is a result of the method.

Workload recipes (paper: Sec. 3.1 simulation recipe, Sec. 3.3 panel shapes):
  * ``panel(n, p, seed, maf=("uniform", .05, .5), miss=.01)``
  * ``phenotype(panel, k_star, effect_var, noise_var, seed)``
  * ``config(i)`` -- the five named workloads (tiny FP64 case, single-solve
    panel, batched CV panel, serving panel, large panel).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

BED_MAGIC = bytes([0x6C, 0x1B, 0x01])
BASE_SEED = 20160803


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` in-tree (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-march=x86-64-v2", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        u64 = ctypes.c_uint64
        u32 = ctypes.c_uint32
        lib.synth_bed_body.argtypes = [P, i64, i64, i64, i64, u64, P, P, u32]
        lib.synth_bed_body.restype = None
        lib.synth_codes.argtypes = [P, i64, P, i64, u64, P, P, u32]
        lib.synth_codes.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Panel:
    """A synthetic genotype panel: n subjects x p SNPs, drawn on demand."""
    n: int
    p: int
    seed: int
    maf: np.ndarray          # float64[p], population alt-allele frequency
    miss: float              # per-call missing probability
    t0: np.ndarray           # uint32[p]  P(code 0) threshold
    t1: np.ndarray           # uint32[p]  P(code 0 or 2) threshold
    tmiss: int               # uint32 threshold on the missingness draw

    @property
    def bed_row_bytes(self) -> int:
        return (self.n + 3) // 4

    def bed_body(self, snp_begin: int = 0, snp_end: int | None = None,
                 row_bytes: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
        """.bed body (no header) for SNPs [snp_begin, snp_end) as uint8[(end-begin)*row_bytes]."""
        snp_end = self.p if snp_end is None else snp_end
        rb = self.bed_row_bytes if row_bytes is None else row_bytes
        assert rb >= self.bed_row_bytes
        m = snp_end - snp_begin
        if out is None:
            out = np.empty(m * rb, dtype=np.uint8)
        assert out.dtype == np.uint8 and out.size >= m * rb and out.flags.c_contiguous
        _load().synth_bed_body(_ptr(out), self.n, snp_begin, snp_end, rb, self.seed,
                               _ptr(self.t0), _ptr(self.t1), self.tmiss)
        return out

    def bed(self) -> np.ndarray:
        """Full .bed file image: magic header + SNP-major body."""
        out = np.empty(3 + self.p * self.bed_row_bytes, dtype=np.uint8)
        out[:3] = np.frombuffer(BED_MAGIC, dtype=np.uint8)
        self.bed_body(out=out[3:])
        return out

    def codes(self, snps) -> np.ndarray:
        """Codes (0 hom-ref, 1 missing, 2 het, 3 hom-alt) of the listed SNPs: int8[m, n]."""
        snps = np.ascontiguousarray(np.asarray(snps, dtype=np.int64))
        out = np.empty((snps.size, self.n), dtype=np.int8)
        if snps.size:
            _load().synth_codes(_ptr(out), self.n, _ptr(snps), snps.size, self.seed,
                                _ptr(self.t0), _ptr(self.t1), self.tmiss)
        return out


def _thresholds(maf: np.ndarray, miss: float):
    q = np.asarray(maf, dtype=np.float64)
    two32 = 4294967296.0
    p0 = (1.0 - q) ** 2
    p01 = p0 + 2.0 * q * (1.0 - q)
    t0 = np.minimum(np.floor(p0 * two32), two32 - 1).astype(np.uint32)
    t1 = np.minimum(np.floor(p01 * two32), two32 - 1).astype(np.uint32)
    tmiss = int(min(np.floor(miss * two32), two32 - 1))
    return t0, t1, tmiss


def panel(n: int, p: int, seed: int, maf=("uniform", 0.05, 0.5), miss: float = 0.01) -> Panel:
    """Draw a panel.  ``maf`` is ("uniform", lo, hi), ("beta", a, b, lo, hi) or an array."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if isinstance(maf, np.ndarray):
        q = maf.astype(np.float64)
    elif maf[0] == "uniform":
        q = rng.uniform(maf[1], maf[2], size=p)
    elif maf[0] == "beta":
        q = np.clip(rng.beta(maf[1], maf[2], size=p), maf[3], maf[4])
    else:
        raise ValueError(maf)
    t0, t1, tmiss = _thresholds(q, miss)
    return Panel(n=n, p=p, seed=seed, maf=q, miss=miss, t0=t0, t1=t1, tmiss=tmiss)


def _pop_standardised(pn: Panel, snps: np.ndarray, rows: np.ndarray | None) -> np.ndarray:
    """Causal columns standardised with the population frequency (missing -> 0)."""
    codes = pn.codes(snps)                                    # [m, n]
    if rows is not None:
        codes = codes[:, rows]
    dose = _DOSE[codes]                                       # missing -> 0 (zeroed below)
    q = pn.maf[snps][:, None]
    z = (dose - 2.0 * q) / np.sqrt(2.0 * q * (1.0 - q))
    z[codes == 1] = 0.0
    return z.T                                                # [n_rows, m]


_DOSE = np.array([0.0, 0.0, 1.0, 2.0])


def phenotype(pn: Panel, k_star: int, effect_var: float, noise_var: float, seed: int,
              rows: np.ndarray | None = None, h2: float | None = None):
    """y = Z_pop beta* + eps over ``rows`` (None = all subjects).

    Returns (y float64[n_rows], causal int64[k_star] ascending, beta* float64[k_star]).
    With ``h2`` given, beta* ~ N(0,1) is rescaled so Var(Z beta*)/(Var(Z beta*)+noise_var) = h2.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    causal = np.sort(rng.choice(pn.p, size=k_star, replace=False)).astype(np.int64)
    beta = rng.normal(0.0, np.sqrt(effect_var), size=k_star)
    z = _pop_standardised(pn, causal, rows)
    signal = z @ beta
    if h2 is not None:
        var_s = float(np.var(signal))
        scale = np.sqrt(h2 / (1.0 - h2) * noise_var / var_s) if var_s > 0 else 0.0
        beta = beta * scale
        signal = signal * scale
    y = signal + rng.normal(0.0, np.sqrt(noise_var), size=signal.shape[0])
    return y, causal, beta


def signal(pn: Panel, causal, beta, rows: np.ndarray | None = None) -> np.ndarray:
    """Z_pop[rows, causal] @ beta: the noise-free part of ``phenotype``'s y."""
    return _pop_standardised(pn, np.asarray(causal, dtype=np.int64), rows) @ np.asarray(beta)


def sim_path(k_true: int, sizes: int = 100, step: int = 2) -> list:
    """Model sizes k0, k0 + step, ... straddling k_true (Sec. 3.1: 100 sizes, step 2)."""
    k0 = max(step, k_true - step * (sizes // 2 - 1))
    return [k0 + step * i for i in range(sizes)]


CONFIGS = {
    # tiny FP64 case the oracle finishes in seconds
    1: dict(name="iht_n1000_p10000_k10", n=1000, p=10000, maf=("uniform", 0.05, 0.5),
            miss=0.01, k_star=10, effect_var=0.25, noise_var=1.0, k=10, tol=1e-4, max_iter=100),
    # single-solve panel (625 MB packed)
    2: dict(name="iht_n5000_p500000_k50", n=5000, p=500000, maf=("uniform", 0.05, 0.5),
            miss=0.01, k_star=50, effect_var=0.1, noise_var=1.0, k=50, tol=1e-4, max_iter=100),
    # batched cross-validation panel (1.5 GB packed): 5 folds x k = 1..20
    3: dict(name="cv_n6000_p1000000_5fold_k1to20", n=6000, p=1000000, maf=("uniform", 0.05, 0.5),
            miss=0.01, k_star=20, effect_var=0.1, noise_var=1.0, folds=5, ks=list(range(1, 21)),
            tol=1e-4, max_iter=100),
    # serving panel (2.5 GB packed)
    4: dict(name="serve_n10000_p1000000", n=10000, p=1000000, maf=("uniform", 0.05, 0.5),
            miss=0.01, requests=2000, tol=1e-4, max_iter=100),
    # large panel (20 GB packed), 32 phenotypes
    5: dict(name="panel_n20000_p4000000_32pheno", n=20000, p=4000000,
            maf=("beta", 0.5, 2.0, 0.01, 0.5), miss=0.02, k_star=100, effect_var=0.1,
            noise_var=1.0, phenotypes=32, k=100, tol=1e-4, max_iter=100),
    # replay of the Sec. 3.1 simulation on a stand-in for its chromosome-1 matrix
    # (5289 subjects x 23 695 SNPs): k_true in {100, 200, 300}, effects
    # N(0, 0.01 / s) for SNR 100 / 50 / 10 / 5 % (s = 1, 2, 10, 20), noise
    # N(0, 0.01), 289 subjects held out, 5-fold CV on the rest over 100 sizes
    6: dict(name="sim_n5289_p23695_ktrue100to300", n=5289, p=23695,
            maf=("beta", 0.5, 2.0, 0.01, 0.5), miss=0.01, k_true=[100, 200, 300],
            snr_s=[1, 2, 10, 20], effect_var=0.01, noise_var=0.01, replicates=10, test=289,
            folds=5, path=100, path_step=2, tol=1e-4, max_iter=100),
}


def config_panel(i: int, n: int | None = None, p: int | None = None) -> Panel:
    c = CONFIGS[i]
    return panel(c["n"] if n is None else n, c["p"] if p is None else p,
                 BASE_SEED + i, maf=c["maf"], miss=c["miss"])


def config_phenotype(i: int, pn: Panel, which: int = 0):
    c = CONFIGS[i]
    return phenotype(pn, c["k_star"], c["effect_var"], c["noise_var"],
                     BASE_SEED + 1000 * i + which)


def cv_folds(n: int, folds: int, seed: int) -> np.ndarray:
    """Fold label in [0, folds) for each subject (random, balanced)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lab = np.arange(n) % folds
    rng.shuffle(lab)
    return lab


def _request_phenotype(args):
    pn, k_star, pseed, rows, h2 = args
    return phenotype(pn, k_star, 1.0, 1.0, pseed, rows=rows, h2=h2)


def serving_requests(pn: Panel, count: int, seed: int, n_lo: int = 2000, n_hi: int = 10000,
                     k_lo: int = 5, k_hi: int = 200, h2_lo: float = 0.1, h2_hi: float = 0.6,
                     workers: int = 1):
    """Serving-stream requests: fresh phenotype, random subject subset, requested k.

    The request parameters come from one sequential stream; the phenotypes
    (own seeds) may be drawn by ``workers`` spawned processes, with identical
    results.  Call it before any CUDA work in the process when workers > 1.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for r in range(count):
        n_rows = int(rng.integers(n_lo, min(n_hi, pn.n) + 1))
        rows = np.sort(rng.choice(pn.n, size=n_rows, replace=False)).astype(np.int32)
        k_star = int(rng.integers(k_lo, k_hi + 1))
        k = int(rng.integers(k_lo, k_hi + 1))
        h2 = float(rng.uniform(h2_lo, h2_hi))
        params.append((rows, k_star, k, h2, seed * 7919 + r))
    jobs = [(pn, ks, ps, rows, h2) for rows, ks, _, h2, ps in params]
    if workers > 1 and count > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            phen = pool.map(_request_phenotype, jobs, chunksize=max(1, count // (4 * workers)))
    else:
        phen = [_request_phenotype(j) for j in jobs]
    out = []
    for (rows, k_star, k, h2, _), (y, causal, beta) in zip(params, phen):
        out.append(dict(rows=rows, y=y, k=k, k_star=k_star, h2=h2, causal=causal))
    return out
