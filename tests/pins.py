"""Pins for the FP64 oracle: checks against things other than the oracle itself.

Each ``pin_*`` takes an oracle library handle (``oracle.load()`` or a build with
a planted mistake) and raises AssertionError when the oracle disagrees with:
  * brute-force pure-Python decoding of the PLINK 2-bit layout (Sec. 2.3.2);
  * exact rational statistics (fractions.Fraction) and numpy's nan-aware
    mean / std (ddof=1) for the per-SNP u, v vectors (Sec. 2.3.2);
  * numpy dense products for the gradient (Eq. normal_grad) and the
    standardisation identity X_st b = X diag(v) b - 1 u^T diag(v) b (Sec. 2.3.2);
  * numpy lexsort for the projection P_{S_k} (Eq. ihta);
  * closed forms of IHT (Sec. 2.2, 2.3.1): single-marker regression at k = 1,
    least squares on the support at a fixed point (Eq. normal_equations), OLS
    when k = p < n, exact recovery of noiseless sparse models, brute force over
    all k-subsets, a monotone objective, |supp beta| <= k, and the sign
    symmetry of allele orientation;
  * an iteration-by-iteration numpy replay of the step size, the backtracking
    rule mu < omega = (1-c) ||d||^2 / ||Z d||^2 and the sufficient decrease it
    implies (Sec. 2.3.1), on instances where the accept decisions depend on c;
  * the stopping rule ||beta+ - beta|| / (||beta|| + 1) < tol recomputed from
    the traced iterates at three scales of y.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np

import oracle

# --------------------------------------------------------------------------
# independent references


def py_decode(body: np.ndarray, n: int, p: int, rb: int) -> np.ndarray:
    """Pure-Python loop decode: sample i of SNP j = bits 2(i%4)..+1 of byte i//4."""
    out = np.empty((p, n), dtype=np.int8)
    b = bytes(body)
    for j in range(p):
        for i in range(n):
            byte = b[j * rb + i // 4]
            out[j, i] = (byte >> (2 * (i % 4))) & 3
    return out


DOSE = {0: 0.0, 2: 1.0, 3: 2.0}


def np_dosage(codes: np.ndarray) -> np.ndarray:
    """Dosage with NaN for missing (code 0 -> 0, 2 -> 1, 3 -> 2, 1 -> NaN)."""
    d = np.full(codes.shape, np.nan)
    for c, x in DOSE.items():
        d[codes == c] = x
    return d


def np_Z(codes: np.ndarray, rows=None) -> np.ndarray:
    """Standardised matrix Z[rows, snps] via numpy nanmean / nanstd(ddof=1); missing -> 0."""
    d = np_dosage(codes)
    if rows is not None:
        d = d[:, rows]
    with np.errstate(invalid="ignore", divide="ignore"):
        m = np.nanmean(d, axis=1, keepdims=True)
        s = np.nanstd(d, axis=1, ddof=1, keepdims=True)
        z = (d - m) / s
    z[~np.isfinite(z)] = 0.0
    z[(s[:, 0] == 0) | ~np.isfinite(s[:, 0]), :] = 0.0
    return z.T


def random_geno(rng, n, p, miss=0.05, rb=None):
    """Random .bed body with genotype frequencies varying per SNP."""
    rb = (n + 3) // 4 if rb is None else rb
    q = rng.uniform(0.05, 0.5, size=p)
    codes = np.empty((p, n), dtype=np.int64)
    for j in range(p):
        pr = np.array([(1 - q[j]) ** 2, 2 * q[j] * (1 - q[j]), q[j] ** 2]) * (1 - miss)
        codes[j] = rng.choice([0, 2, 3, 1], size=n, p=np.append(pr, miss))
    body = np.zeros(p * rb, dtype=np.uint8)
    for j in range(p):
        for i in range(n):
            body[j * rb + i // 4] |= codes[j, i] << (2 * (i % 4))
    return oracle.Geno(body, n, p, rb), codes.astype(np.int8)


def geno_from_codes(codes: np.ndarray) -> oracle.Geno:
    p, n = codes.shape
    rb = (n + 3) // 4
    body = np.zeros(p * rb, dtype=np.uint8)
    for j in range(p):
        for i in range(n):
            body[j * rb + i // 4] |= int(codes[j, i]) << (2 * (i % 4))
    return oracle.Geno(body, n, p, rb)


def lstsq_obj(Z, y, cols):
    """Least-squares refit on the given columns: (coef, 1/2 ||y - Z_S coef||^2)."""
    if len(cols) == 0:
        return np.zeros(0), 0.5 * float(y @ y)
    A = Z[:, list(cols)]
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    res = y - A @ coef
    return coef, 0.5 * float(res @ res)


# --------------------------------------------------------------------------
# pins


def pin_decode(lib):
    rng = np.random.default_rng(11)
    for n in (1, 2, 3, 4, 5, 7, 13, 33):
        for extra in (0, 5):
            rb = (n + 3) // 4 + extra
            p = 6
            body = rng.integers(0, 256, size=p * rb, dtype=np.uint8)
            got = oracle.decode(oracle.Geno(body, n, p, rb), lib=lib)
            assert np.array_equal(got, py_decode(body, n, p, rb)), f"decode n={n} rb={rb}"


def pin_counts_stats(lib):
    rng = np.random.default_rng(12)
    for n, miss in ((9, 0.1), (37, 0.02), (64, 0.3)):
        G, codes = random_geno(rng, n, 25, miss=miss)
        for rows in (None, np.sort(rng.choice(n, size=max(3, n // 2), replace=False))):
            c, u, v = oracle.counts(G, rows, lib=lib)
            sub = codes if rows is None else codes[:, rows]
            want = np.stack([np.bincount(sub[j], minlength=4) for j in range(G.p)])
            assert np.array_equal(c, want), "counts"
            d = np_dosage(sub)
            with np.errstate(invalid="ignore", divide="ignore"):
                m = np.nanmean(d, axis=1)
                s = np.nanstd(d, axis=1, ddof=1)
            ok = np.isfinite(s) & (s > 0)
            assert np.allclose(u[ok], m[ok], rtol=1e-14, atol=0), "mean u"
            assert np.allclose(v[ok], 1.0 / s[ok], rtol=1e-13, atol=0), "inverse sd v"
            assert np.all(v[~ok] == 0.0), "v = 0 for monomorphic columns"


def pin_stats_exact(lib):
    """u and v against exact rational arithmetic (v within 2 ulp of 1/sqrt(var))."""
    codes = np.array([[0, 2, 3, 1, 2, 0, 3],      # mixed, one missing
                      [3, 3, 3, 3, 1, 3, 3],      # monomorphic among observed -> v = 0
                      [1, 1, 1, 1, 1, 1, 2],      # one observed call -> v = 0
                      [2, 2, 0, 0, 3, 1, 1]], dtype=np.int8)
    G = geno_from_codes(codes)
    _, u, v = oracle.counts(G, lib=lib)
    for j in range(codes.shape[0]):
        xs = [Fraction(int(DOSE[c])) for c in codes[j] if c != 1]
        m = sum(xs, Fraction(0)) / len(xs) if xs else Fraction(0)
        assert u[j] == float(m), f"u[{j}]"
        if len(xs) >= 2:
            var = sum(((x - m) ** 2 for x in xs), Fraction(0)) / (len(xs) - 1)
        else:
            var = Fraction(0)
        if var == 0:
            assert v[j] == 0.0, f"v[{j}] should be 0"
        else:
            want = 1.0 / np.sqrt(float(var))
            assert abs(v[j] - want) <= 4e-16 * want, f"v[{j}]"


def pin_gradient(lib):
    rng = np.random.default_rng(13)
    for n, p in ((50, 30), (123, 17)):
        G, codes = random_geno(rng, n, p, miss=0.05)
        for rows in (None, np.sort(rng.choice(n, size=n - 7, replace=False))):
            nr = n if rows is None else rows.size
            r = rng.normal(size=nr)
            g = oracle.gradient(G, r, rows, lib=lib)
            Z = np_Z(codes, rows)
            want = Z.T @ r
            assert np.max(np.abs(g - want)) <= 1e-12 * np.max(np.abs(want)), "g = Z^T r"
            # centring: a constant residual has zero gradient
            g1 = oracle.gradient(G, np.ones(nr), rows, lib=lib)
            assert np.max(np.abs(g1)) <= 1e-11, "columns centred"
            # unit variance with the (n_obs - 1) denominator: z_j^T z_j = n_obs - 1
            sub = codes if rows is None else codes[:, rows]
            for j in range(0, p, 5):
                gz = oracle.gradient(G, Z[:, j], rows, lib=lib)[j]
                n_obs = int(np.sum(sub[j] != 1))
                if np.any(Z[:, j] != 0):
                    assert abs(gz - (n_obs - 1)) <= 1e-10 * n_obs, "z^T z = n_obs - 1"


def pin_identity(lib):
    """X_st b = X diag(v) b - 1 u^T diag(v) b on mean-imputed X (Sec. 2.3.2)."""
    rng = np.random.default_rng(14)
    G, codes = random_geno(rng, 71, 23, miss=0.08)
    _, u, v = oracle.counts(G, lib=lib)
    X = np_dosage(codes).T                       # n x p, NaN for missing
    X = np.where(np.isnan(X), u[None, :], X)     # mean imputation
    cols = np.array([0, 3, 4, 9, 22], dtype=np.int32)
    b = rng.normal(size=cols.size)
    want = X[:, cols] @ (v[cols] * b) - np.ones(G.n) * (u[cols] @ (v[cols] * b))
    got = oracle.zmul(G, cols, b, lib=lib)
    assert np.max(np.abs(got - want)) <= 1e-12 * (1 + np.max(np.abs(want))), "identity"
    # and against the numpy-standardised matrix
    Z = np_Z(codes)
    assert np.allclose(got, Z[:, cols] @ b, rtol=1e-12, atol=1e-12), "zmul vs numpy"
    # held-out rows with training statistics
    tr = np.arange(0, G.n, 2)
    te = np.arange(1, G.n, 2)
    _, ut, vt = oracle.counts(G, tr, lib=lib)
    got_te = oracle.zmul(G, cols, b, rows=te, u=ut, v=vt, lib=lib)
    d = np_dosage(codes)[:, te]
    zt = np.where(np.isnan(d), 0.0, vt[:, None] * (d - ut[:, None])).T
    assert np.allclose(got_te, zt[:, cols] @ b, rtol=1e-12, atol=1e-12), "held-out rows"


def pin_topk(lib):
    rng = np.random.default_rng(15)
    for p, k in ((10, 1), (10, 10), (100, 7), (1000, 37)):
        for kind in ("real", "ties"):
            w = rng.normal(size=p) if kind == "real" else rng.integers(-3, 4, size=p).astype(float)
            got = oracle.topk(w, k, lib=lib)
            want = np.lexsort((np.arange(p), -np.abs(w)))[:k]
            assert np.array_equal(got, want), f"topk {kind} p={p} k={k}"


def _panel(seed, n, p, miss=0.01):
    rng = np.random.default_rng(seed)
    G, codes = random_geno(rng, n, p, miss=miss)
    return rng, G, codes


def pin_k1_marginal(lib):
    """k = 1: S^0 = argmax |z_j^T y| and beta = z_j^T y / z_j^T z_j (marginal regression)."""
    for seed in (21, 22, 23):
        rng, G, codes = _panel(seed, 200, 60)
        y = rng.normal(size=G.n)
        Z = np_Z(codes)
        f = oracle.iht(G, y, 1, max_iter=1, lib=lib)
        s = Z.T @ y
        j = int(np.lexsort((np.arange(G.p), -np.abs(s)))[0])
        assert f.trace["supp"][0, 0] == j, "k=1 first support is the single-marker scan"
        want = s[j] / (Z[:, j] @ Z[:, j])
        assert abs(f.beta[j] - want) <= 1e-12 * abs(want), "k=1 step solves the marginal LS"


def pin_fixed_point(lib):
    """At convergence with a stable support, beta_S solves the normal equations on S."""
    for seed in (31, 32, 33, 34):
        rng, G, codes = _panel(seed, 300, 80)
        Z = np_Z(codes)
        true = rng.choice(G.p, size=4, replace=False)
        y = Z[:, true] @ rng.normal(0, 1.0, size=4) + rng.normal(size=G.n)
        f = oracle.iht(G, y, 4, tol=1e-11, max_iter=5000, lib=lib)
        assert f.status == oracle.OK
        coef, obj = lstsq_obj(Z, y, f.support)
        assert np.allclose(f.beta[f.support], coef, rtol=1e-7, atol=1e-9), "normal equations"
        assert abs(f.objective - obj) <= 1e-9 * obj


def pin_full_ols(lib):
    """k = p < n: normalized steepest descent converges to the OLS fit."""
    rng, G, codes = _panel(41, 120, 6, miss=0.0)
    Z = np_Z(codes)
    y = Z @ rng.normal(size=6) + rng.normal(size=G.n)
    f = oracle.iht(G, y, 6, tol=1e-13, max_iter=20000, lib=lib)
    coef, _ = lstsq_obj(Z, y, range(6))
    assert np.allclose(f.beta, coef, rtol=1e-8, atol=1e-10), "OLS"


def pin_noiseless(lib):
    """y = Z_S b exactly, well-separated effects: exact recovery of S and b."""
    for seed in (51, 52):
        rng, G, codes = _panel(seed, 400, 50, miss=0.0)
        Z = np_Z(codes)
        S = np.sort(rng.choice(G.p, size=3, replace=False))
        b = np.array([3.0, -2.5, 2.0])
        y = Z[:, S] @ b
        f = oracle.iht(G, y, 3, tol=1e-12, max_iter=5000, lib=lib)
        assert np.array_equal(np.sort(f.support), S), "support recovery"
        assert np.allclose(f.beta[S], b, rtol=1e-7, atol=1e-9), "coefficients"
        assert f.objective <= 1e-12 * float(y @ y)


def pin_bruteforce(lib):
    """f(beta_IHT) >= min over all k-subsets of the LS objective; equality on strong signals."""
    for seed in (61, 62, 63, 64, 65):
        rng, G, codes = _panel(seed, 40, 12, miss=0.0)
        Z = np_Z(codes)
        for k in (1, 2, 3):
            for strong in (False, True):
                if strong:
                    S = rng.choice(G.p, size=k, replace=False)
                    y = Z[:, S] @ (rng.choice([-1, 1], size=k) * rng.uniform(4, 6, size=k)) \
                        + 0.3 * rng.normal(size=G.n)
                else:
                    y = rng.normal(size=G.n)
                best = min(lstsq_obj(Z, y, c)[1] for c in itertools.combinations(range(G.p), k))
                f = oracle.iht(G, y, k, tol=1e-12, max_iter=5000, lib=lib)
                assert f.objective >= best - 1e-9 * (1 + best), "objective below the subset optimum"
                if strong:
                    assert abs(f.objective - best) <= 1e-7 * (1 + best), "strong signal: optimum"


def pin_invariants(lib):
    """Monotone objective, |supp beta| <= k, sorted support, accepted steps satisfy mu < omega."""
    for seed in (71, 72, 73):
        rng, G, codes = _panel(seed, 150, 300, miss=0.02)
        Z = np_Z(codes)
        S = rng.choice(G.p, size=8, replace=False)
        y = Z[:, S] @ rng.normal(0, 0.5, size=8) + rng.normal(size=G.n)
        for k in (1, 5, 8, 20):
            f = oracle.iht(G, y, k, tol=1e-8, max_iter=300, lib=lib)
            obj = np.concatenate([[0.5 * float(y @ y)], f.trace["objective"]])
            assert np.all(np.diff(obj) <= 1e-12 * obj[:-1]), "monotone objective"
            assert np.count_nonzero(f.beta) <= k
            assert np.all(np.diff(f.support) > 0) and f.support.size == k
            off = np.setdiff1d(np.arange(G.p), f.support)
            assert np.all(f.beta[off] == 0.0)
            ch = (f.trace["changed"] == 1) & (f.trace["backtracks"] < 50)
            assert np.all(f.trace["mu"][ch] < f.trace["omega"][ch]), "accepted mu < omega"
            # objective reported = 1/2 ||y - Z beta||^2 from scratch
            res = y - Z @ f.beta
            assert abs(f.objective - 0.5 * res @ res) <= 1e-10 * f.objective


def pin_orientation(lib):
    """Swapping hom-ref and hom-alt codes flips z: same support, beta -> -beta."""
    rng, G, codes = _panel(81, 200, 40, miss=0.03)
    Z = np_Z(codes)
    y = Z[:, [3, 17]] @ np.array([1.5, -1.0]) + rng.normal(size=G.n)
    flipped = codes.copy()
    flipped[codes == 0] = 3
    flipped[codes == 3] = 0
    G2 = geno_from_codes(flipped)
    a = oracle.iht(G, y, 2, tol=1e-10, max_iter=1000, lib=lib)
    b = oracle.iht(G2, y, 2, tol=1e-10, max_iter=1000, lib=lib)
    assert np.array_equal(a.support, b.support)
    assert np.allclose(a.beta, -b.beta, rtol=1e-9, atol=1e-12)


def pin_cv(lib):
    """Cross-validation (Sec. 2.4) against numpy: each partition's rows
    standardised with the numpy statistics of the other partitions' rows,
    predictions from the fold fits, each partition's MSE, their mean per model
    size (unequal partitions, so a pooled MSE would differ), the first least
    size and the refit on the labelled rows; subjects labelled -1 (a held-out
    set) take part in nothing."""
    rng, G, codes = _panel(41, 150, 40, miss=0.03)
    y = np_Z(codes)[:, [3, 17, 30]] @ np.array([0.8, -0.6, 0.7]) + rng.normal(size=G.n)
    q, ks = 3, [1, 2, 3, 5]
    fold = rng.permutation(np.repeat(np.arange(-1, q), [12, 40, 45, 53]))    # 12 held out
    res = oracle.cv(G, y, fold, q, ks, lib=lib)
    d = np_dosage(codes)                                        # p x n, NaN = missing
    want = np.zeros((q, len(ks)))
    for f in range(q):
        tr, te = (fold != f) & (fold >= 0), fold == f
        with np.errstate(invalid="ignore", divide="ignore"):
            m = np.nanmean(d[:, tr], axis=1)
            s = np.nanstd(d[:, tr], axis=1, ddof=1)
            zt = (d[:, te] - m[:, None]) / s[:, None]
        zt[~np.isfinite(zt)] = 0.0
        zt[(s == 0) | ~np.isfinite(s), :] = 0.0
        for t, k in enumerate(ks):
            fit = res.fits[f][t]
            alone = oracle.iht(G, y[tr], k, rows=np.flatnonzero(tr).astype(np.int32), trace=False,
                               lib=lib)
            assert np.array_equal(fit.beta, alone.beta), "fold fit is the training-rows solve"
            want[f, t] = np.mean((y[te] - zt.T @ fit.beta) ** 2)
    assert np.allclose(res.mse_fold, want, rtol=1e-10, atol=0), "partition MSE"
    assert np.allclose(res.mse, want.mean(axis=0), rtol=1e-10, atol=0), "MSE averaged over partitions"
    assert res.k_best == ks[int(np.argmin(want.mean(axis=0)))], "least averaged MSE"
    inside = np.flatnonzero(fold >= 0).astype(np.int32)
    refit = oracle.iht(G, y[inside], res.k_best, rows=inside, trace=False, lib=lib)
    assert np.array_equal(res.fit.beta, refit.beta), "refit on the labelled rows at k_best"



def _np_topk(w, k):
    """P_{S_k} by numpy: the k largest |w|, ties to the lower index, ascending."""
    return np.sort(np.lexsort((np.arange(w.size), -np.abs(w)))[:k])


def _np_iteration(Z, y, beta, S, k, c, kappa, max_bt):
    """One IHT iteration in numpy (Sec. 2.2, 2.3.1): normalized step on S,
    projection, and the backtracking rule shrink-while mu >= (1-c) rho,
    rho = ||d||^2 / ||Z d||^2, applied when the support changes.  Returns
    (S+, beta+, accepted mu, shrinks, decisions) where decisions lists
    (mu, rho) for every omega check made."""
    g = Z.T @ (y - Z @ beta)
    mu = (g[S] @ g[S]) / np.sum((Z[:, S] @ g[S]) ** 2)
    decisions = []
    for j in range(max_bt + 1):
        w = beta + mu * g
        Sp = _np_topk(w, k)
        bp = np.zeros_like(beta)
        bp[Sp] = w[Sp]
        if np.array_equal(Sp, S):
            return Sp, bp, mu, j, decisions
        d = bp - beta
        rho = (d @ d) / np.sum((Z @ d) ** 2)
        decisions.append((mu, rho))
        if mu < (1 - c) * rho or j == max_bt:
            return Sp, bp, mu, j, decisions
        mu /= kappa
    raise AssertionError("unreachable")


def pin_backtracking_replay(lib):
    """Every iteration replayed in numpy from the oracle's previous iterate: the
    step size, each backtracking decision and the accepted support, beta and
    shrink count agree, and the omega the oracle reports is (1-c) rho of its
    accepted candidate (Sec. 2.3.1).  With c = 0.3 many decisions fall where
    mu < (1-c) rho, mu < rho and mu < (1+c) rho disagree, so a dropped or
    flipped (1-c) factor changes a decision; the pin asserts such decisions
    occurred.  Accepted steps also satisfy the sufficient decrease that the
    rule guarantees: f(beta) - f(beta+) > c ||d||^2 / (2 mu), from
    g^T d >= ||d||^2 / (2 mu) (beta+ is the best k-sparse approximation of
    beta + mu g) and ||Z d||^2 < (1-c) ||d||^2 / mu."""
    cases = [(70, 12, 0.3), (71, 5, 0.3), (74, 12, 0.3), (70, 12, 0.01), (71, 12, 0.01)]
    sensitive = 0
    for seed, k, c in cases:
        rng, G, codes = _panel(seed, 150, 300, miss=0.02)
        Z = np_Z(codes)
        causal = rng.choice(G.p, size=8, replace=False)
        y = Z[:, causal] @ rng.normal(0, 0.5, size=8) + rng.normal(size=G.n)
        f = oracle.iht(G, y, k, c=c, tol=1e-4, max_iter=200, lib=lib)
        assert f.iterations >= 3
        beta = np.zeros(G.p)
        S = _np_topk(Z.T @ y, k)
        for t in range(f.iterations):
            Sp, bp, mu, bt, dec = _np_iteration(Z, y, beta, S, k, c, 2.0, 50)
            assert np.array_equal(Sp, f.trace["supp"][t]), f"support at iteration {t}"
            assert np.allclose(bp[Sp], f.trace["beta"][t], rtol=1e-9, atol=1e-12), f"beta at {t}"
            assert bt == f.trace["backtracks"][t], f"shrinks at iteration {t}"
            assert abs(mu - f.trace["mu"][t]) <= 1e-9 * mu, f"step size at iteration {t}"
            if dec:
                m_, rho = dec[-1]
                assert abs(f.trace["omega"][t] - (1 - c) * rho) <= 1e-9 * rho, f"omega at {t}"
                for m_, rho in dec:
                    a = m_ < (1 - c) * rho
                    sensitive += a != (m_ < rho) or a != (m_ < (1 + c) * rho)
                if bt < 50:
                    d = bp - beta
                    f0 = 0.5 * np.sum((y - Z @ beta) ** 2)
                    f1 = 0.5 * np.sum((y - Z @ bp) ** 2)
                    assert f0 - f1 > c * (d @ d) / (2 * mu) * (1 - 1e-9), f"decrease at {t}"
            beta, S = bp, Sp
    assert sensitive >= 10, "instances must exercise decisions that depend on c"


def pin_convergence_rule(lib):
    """The solve stops at the first iteration with ||beta+ - beta|| / (||beta|| + 1)
    < tol, recomputed in numpy from the traced iterates, and not before.  The
    same problem is solved with y scaled by 1e-3, 1 and 1e3 (IHT's supports and
    step sizes are scale-invariant; only the stopping test sees the scale): at
    1e3 the stop happens while ||beta+ - beta|| itself is still >= tol, at 1e-3
    while ||beta+ - beta|| / ||beta|| is still >= tol, so a test without the
    +1 or with a plain relative denominator stops at another iteration."""
    rng, G, codes = _panel(72, 150, 300, miss=0.02)
    Z = np_Z(codes)
    causal = rng.choice(G.p, size=8, replace=False)
    y0 = Z[:, causal] @ rng.normal(0, 0.5, size=8) + rng.normal(size=G.n)
    tol = 1e-4
    stops = []
    for s in (1e-3, 1.0, 1e3):
        f = oracle.iht(G, s * y0, 12, tol=tol, max_iter=300, lib=lib)
        assert f.status == oracle.OK
        prev = np.zeros(G.p)
        steps, dn, bn = [], [], []
        for t in range(f.iterations):
            cur = np.zeros(G.p)
            cur[f.trace["supp"][t]] = f.trace["beta"][t]
            dn.append(np.linalg.norm(cur - prev))
            bn.append(np.linalg.norm(prev))
            steps.append(dn[-1] / (bn[-1] + 1.0))
            prev = cur
        steps = np.array(steps)
        assert np.all(steps[:-1] >= tol), f"scale {s}: stopped late"
        assert steps[-1] < tol, f"scale {s}: stopped early"
        stops.append((s, dn[-1], bn[-1]))
    s, d, b = stops[2]
    assert d >= tol, "the 1e3 instance must separate the +1 rule from an absolute test"
    s, d, b = stops[0]
    assert d / b >= tol, "the 1e-3 instance must separate the +1 rule from a relative test"



def _np_htp_iteration(Z, y, beta, S, k, c, kappa, max_bt):
    """One HTP iteration in numpy (Sec. 2.2 and the step-size reading R11):
    the normalized step over Gamma = the k largest |g|, IHT's projection and
    backtracking rule on the candidate, then least squares on S+ (numpy
    lstsq).  Returns (S+, beta+, mu, shrinks)."""
    g = Z.T @ (y - Z @ beta)
    gam = _np_topk(g, k)
    mu = (g[gam] @ g[gam]) / np.sum((Z[:, gam] @ g[gam]) ** 2)
    for j in range(max_bt + 1):
        w = beta + mu * g
        Sp = _np_topk(w, k)
        if np.array_equal(Sp, S):
            break
        bp = np.zeros_like(beta)
        bp[Sp] = w[Sp]
        d = bp - beta
        rho = (d @ d) / np.sum((Z @ d) ** 2)
        if mu < (1 - c) * rho or j == max_bt:
            break
        mu /= kappa
    out = np.zeros_like(beta)
    out[Sp] = np.linalg.lstsq(Z[:, Sp], y, rcond=None)[0]
    return Sp, out, mu, j


def pin_htp_replay(lib):
    """HTP, iteration by iteration against numpy: the step over the k largest
    |g| (after a refit g vanishes on S), the backtracking decisions on the
    projected candidate, the support, beta+ = least squares on S+ (Eq.
    normal_equations) and the stopping rule; the objective never increases."""
    for seed, k, c in ((70, 5, 0.01), (71, 12, 0.01), (72, 12, 0.3), (74, 8, 0.3), (79, 5, 0.3)):
        rng, G, codes = _panel(seed, 150, 300, miss=0.02)
        Z = np_Z(codes)
        causal = rng.choice(G.p, size=8, replace=False)
        y = Z[:, causal] @ rng.normal(0, 0.5, size=8) + rng.normal(size=G.n)
        f = oracle.iht(G, y, k, c=c, tol=1e-10, max_iter=100, variant="htp", lib=lib)
        assert f.status == oracle.OK and f.iterations >= 2
        beta = np.zeros(G.p)
        S = _np_topk(Z.T @ y, k)
        fprev = 0.5 * float(y @ y)
        for t in range(f.iterations):
            Sp, bp, mu, bt = _np_htp_iteration(Z, y, beta, S, k, c, 2.0, 50)
            assert np.array_equal(Sp, f.trace["supp"][t]), f"support at iteration {t}"
            assert np.allclose(bp[Sp], f.trace["beta"][t], rtol=1e-8, atol=1e-10), f"refit at {t}"
            assert abs(mu - f.trace["mu"][t]) <= 1e-8 * mu, f"step size at iteration {t}"
            assert bt == f.trace["backtracks"][t], f"shrinks at iteration {t}"
            step = np.linalg.norm(bp - beta) / (np.linalg.norm(beta) + 1.0)
            assert (step < 1e-10) == (t == f.iterations - 1), f"stopping rule at {t}"
            fcur = 0.5 * float(np.sum((y - Z @ bp) ** 2))
            assert abs(f.trace["objective"][t] - fcur) <= 1e-9 * fcur
            assert fcur <= fprev * (1 + 1e-12), f"objective increased at {t}"
            beta, S, fprev = bp, Sp, fcur


def pin_htp_closed_forms(lib):
    """HTP on tiny inputs: never below the best k-subset least-squares fit,
    equal to it on strong signals; k = p < n gives OLS after one step and
    stops at the next; a duplicated column and a monomorphic column among the
    predictors leave the fitted values those of numpy's least squares, with
    coefficient 0 on the later duplicate and on the constant column."""
    for seed in (61, 62, 63):
        rng, G, codes = _panel(seed, 40, 12, miss=0.0)
        Z = np_Z(codes)
        for k in (1, 2, 3):
            for strong in (False, True):
                if strong:
                    S = rng.choice(G.p, size=k, replace=False)
                    y = Z[:, S] @ (rng.choice([-1, 1], size=k) * rng.uniform(4, 6, size=k)) \
                        + 0.3 * rng.normal(size=G.n)
                else:
                    y = rng.normal(size=G.n)
                best = min(lstsq_obj(Z, y, cc)[1] for cc in itertools.combinations(range(G.p), k))
                f = oracle.iht(G, y, k, tol=1e-12, max_iter=500, variant="htp", lib=lib)
                assert f.objective >= best - 1e-9 * (1 + best), "HTP below the subset optimum"
                if strong:
                    assert abs(f.objective - best) <= 1e-9 * (1 + best), "strong signal: optimum"
    rng, G, codes = _panel(41, 120, 6, miss=0.0)
    Z = np_Z(codes)
    y = Z @ rng.normal(size=6) + rng.normal(size=G.n)
    f = oracle.iht(G, y, 6, tol=1e-12, max_iter=50, variant="htp", lib=lib)
    coef, _ = lstsq_obj(Z, y, range(6))
    assert np.allclose(f.trace["beta"][0], coef, rtol=1e-9, atol=1e-12), "k = p: OLS in one step"
    assert f.iterations == 2 and f.status == oracle.OK
    rng = np.random.default_rng(91)
    _, codes = random_geno(rng, 90, 10, miss=0.0)
    codes[7] = codes[2]                                   # column 7 duplicates column 2
    codes[5] = 3                                          # column 5 is monomorphic
    G = geno_from_codes(codes)
    Z = np_Z(codes)
    y = Z[:, [2, 4]] @ np.array([1.5, -1.0]) + 0.5 * rng.normal(size=G.n)
    f = oracle.iht(G, y, 10, tol=1e-12, max_iter=50, variant="htp", lib=lib)
    fit = Z @ f.beta
    want = Z @ np.linalg.lstsq(Z, y, rcond=None)[0]
    assert np.allclose(fit, want, rtol=1e-9, atol=1e-9), "fitted values of the full refit"
    assert f.beta[7] == 0.0 and f.beta[5] == 0.0, "dependent and zero columns get 0"


def _cov_panel(seed):
    rng, G, codes = _panel(seed, 200, 60, miss=0.02)
    cov = np.vstack([rng.normal(size=G.n), (rng.random(G.n) < 0.4).astype(float),
                     rng.gamma(2.0, size=G.n), np.full(G.n, 3.0)])     # last one constant
    return rng, G, codes, cov


def _np_cov_z(cov, rows=None):
    c = cov if rows is None else cov[:, rows]
    m = c.mean(axis=1, keepdims=True)
    s = c.std(axis=1, ddof=1, keepdims=True)
    with np.errstate(invalid="ignore", divide="ignore"):
        z = np.where(s > 0, (c - m) / s, 0.0)
    return z.T


def pin_cov_stats(lib):
    """Covariate mean / inverse SD (reading R13) against numpy, with a row subset
    and a constant column (inverse SD 0)."""
    rng, G, codes, cov = _cov_panel(83)
    for rows in (None, np.sort(rng.choice(G.n, size=77, replace=False))):
        cu, cv = oracle.cov_stats(cov, G.n, rows, lib=lib)
        c = cov if rows is None else cov[:, rows]
        assert np.allclose(cu, c.mean(axis=1), rtol=1e-13, atol=1e-13)
        sd = c.std(axis=1, ddof=1)
        assert np.allclose(cv[:3], 1.0 / sd[:3], rtol=1e-12) and cv[3] == 0.0


def pin_cov_design(lib):
    """IHT with covariates is IHT on the design [Z | C_std] (covariates standardised
    over the used rows, appended after the SNPs, counted in k): each iteration
    replayed in numpy on that matrix; with a row subset too; and at a fixed
    point beta solves the normal equations on its support."""
    rng, G, codes, cov = _cov_panel(84)
    for rows in (None, np.sort(rng.choice(G.n, size=170, replace=False))):
        Z = np.hstack([np_Z(codes, rows), _np_cov_z(cov, rows)])
        nr = Z.shape[0]
        y = Z[:, [4, 11, G.p, G.p + 2]] @ np.array([0.8, -0.6, 1.5, 0.7]) + rng.normal(size=nr)
        for k in (3, 6):
            f = oracle.iht(G, y, k, rows=rows, cov=cov, tol=1e-4, max_iter=200, lib=lib)
            assert np.any(f.support >= G.p), "a covariate enters the support"
            beta = np.zeros(G.p + cov.shape[0])
            S = _np_topk(Z.T @ y, k)
            for t in range(f.iterations):
                Sp, bp, mu, bt, _ = _np_iteration(Z, y, beta, S, k, 0.01, 2.0, 50)
                assert np.array_equal(Sp, f.trace["supp"][t]), f"support at iteration {t}"
                assert np.allclose(bp[Sp], f.trace["beta"][t], rtol=1e-9, atol=1e-12)
                beta, S = bp, Sp
        f = oracle.iht(G, y, 4, rows=rows, cov=cov, tol=1e-12, max_iter=5000, lib=lib)
        coef, obj = lstsq_obj(Z, y, f.support)
        assert np.allclose(f.beta[f.support], coef, rtol=1e-7, atol=1e-9), "normal equations"


ALL_PINS = [pin_decode, pin_counts_stats, pin_stats_exact, pin_gradient, pin_identity, pin_topk,
            pin_k1_marginal, pin_fixed_point, pin_full_ols, pin_noiseless, pin_bruteforce,
            pin_invariants, pin_orientation, pin_cv, pin_backtracking_replay,
            pin_convergence_rule, pin_htp_replay, pin_htp_closed_forms, pin_cov_stats,
            pin_cov_design]
