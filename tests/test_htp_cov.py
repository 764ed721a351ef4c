"""HTP and nongenetic covariates on the GPU against the FP64 oracle (needs a B300).

Bars as in test_gpu_parity: supports equal while the oracle certifies the
selection (gap between the k-th and (k+1)-th |w| above the FP32 gradient error,
no backtracking decision within 1e-3 of its threshold); beta within 1e-4
relative (HTP's beta is an FP64 least-squares fit on the support, so it is
compared at 1e-9 once the supports agree); objective within 1e-6.
"""
import numpy as np
import pytest

import oracle
import synth
from pins import np_Z, random_geno, geno_from_codes
from test_gpu_parity import compare_fits, rel_err

pytestmark = pytest.mark.gpu

MAGIC = np.array([0x6C, 0x1B, 0x01], dtype=np.uint8)


@pytest.fixture(scope="module")
def iht():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_01398_b300 as m
    return m


@pytest.fixture(scope="module")
def ctx(iht):
    return iht.Context(0)


def load(iht, ctx, G):
    return iht.Dataset(ctx, np.concatenate([MAGIC, G.body]), G.n, G.p)


def check_htp_fit(fo, fg, k):
    n = compare_fits(fo, fg, k)
    for t in range(n):                      # FP64 refit on equal supports
        assert rel_err(fg.trace["beta"][t], fo.trace["beta"][t]) <= 1e-9, f"refit at {t}"
    return n


def test_htp_parity_config1(iht, ctx):
    pn = synth.config_panel(1)
    G = oracle.Geno.from_bed(pn.bed(), pn.n, pn.p)
    ds = load(iht, ctx, G)
    y, _, _ = synth.config_phenotype(1, pn)
    fo = oracle.iht(G, y, 10, variant="htp")
    for impl in (1, 2):
        fg = iht.iht_fit_trace(ds, y, 10, grad_impl=impl, variant="htp")
        assert check_htp_fit(fo, fg, 10) == fo.iterations
        assert fg.iterations == fo.iterations and fg.status == fo.status
        assert np.array_equal(fg.support, fo.support)
    plain = iht.iht_fit(ds, y, 10, variant="htp")        # untraced path: same result
    assert np.array_equal(plain.beta, fg.beta) and plain.iterations == fg.iterations


@pytest.mark.parametrize("seed", range(5))
def test_htp_small_panels(iht, ctx, seed):
    rng = np.random.default_rng(300 + seed)
    n = [150, 333, 401, 1000, 257][seed]
    p = [300, 500, 1201, 3000, 90][seed]
    k = [5, 12, 30, 20, 9][seed]
    c = [0.01, 0.3, 0.01, 0.3, 0.01][seed]
    G, codes = random_geno(rng, n, p, miss=0.02)
    ds = load(iht, ctx, G)
    rows = None if seed % 2 == 0 else np.sort(rng.choice(n, size=n - 11, replace=False))
    nr = n if rows is None else rows.size
    Z = np_Z(codes, rows)
    causal = rng.choice(p, size=min(k, p), replace=False)
    y = Z[:, causal] @ rng.normal(0, 0.5, size=causal.size) + rng.normal(size=nr) + 0.5
    fo = oracle.iht(G, y, k, rows=rows, c=c, max_iter=60, tol=1e-8, variant="htp")
    fg = iht.iht_fit_trace(ds, y, k, rows=rows, c=c, max_iter=60, tol=1e-8, variant="htp")
    got = check_htp_fit(fo, fg, k)
    print(f"certified {got} of {fo.iterations} iterations")
    assert got >= 1
    obj = np.concatenate([[0.5 * float(y @ y)], fg.trace["objective"]])
    assert np.all(np.diff(obj) <= 1e-9 * obj[:-1]), "monotone objective"
    # the result is the least-squares fit on its support
    coef = np.linalg.lstsq(Z[:, fg.support], y, rcond=None)[0]
    assert rel_err(fg.beta[fg.support], coef) <= 1e-8


def test_htp_k_equals_p_and_dependent_columns(iht, ctx):
    rng = np.random.default_rng(41)
    G, codes = random_geno(rng, 120, 6, miss=0.0)
    ds = load(iht, ctx, G)
    Z = np_Z(codes)
    y = Z @ rng.normal(size=6) + rng.normal(size=120)
    fg = iht.iht_fit(ds, y, 6, tol=1e-12, variant="htp")
    assert rel_err(fg.beta, np.linalg.lstsq(Z, y, rcond=None)[0]) <= 1e-10
    assert fg.iterations == 2
    _, codes = random_geno(np.random.default_rng(91), 90, 10, miss=0.0)
    codes[7] = codes[2]                                   # duplicate of column 2
    codes[5] = 3                                          # monomorphic
    G2 = geno_from_codes(codes)
    ds2 = load(iht, ctx, G2)
    Z = np_Z(codes)
    y = Z[:, [2, 4]] @ np.array([1.5, -1.0]) + 0.5 * np.random.default_rng(1).normal(size=90)
    fg = iht.iht_fit(ds2, y, 10, tol=1e-12, variant="htp")
    fo = oracle.iht(G2, y, 10, tol=1e-12, variant="htp", trace=False)
    assert fg.beta[7] == 0.0 and fg.beta[5] == 0.0
    assert np.allclose(Z @ fg.beta, Z @ fo.beta, rtol=1e-9, atol=1e-9)


def cov_panel(seed, n=600, p=2000):
    rng = np.random.default_rng(seed)
    G, codes = random_geno(rng, n, p, miss=0.02)
    cov = np.vstack([rng.normal(size=n), (rng.random(n) < 0.4).astype(float),
                     rng.gamma(2.0, size=n), np.full(n, 3.0)])
    return rng, G, codes, cov


@pytest.mark.parametrize("variant", ["iht", "htp"])
@pytest.mark.parametrize("subset", [False, True])
def test_covariates_parity(iht, ctx, variant, subset):
    rng, G, codes, cov = cov_panel(500 + subset)
    ds = load(iht, ctx, G)
    ds.set_covariates(cov)
    rows = np.sort(rng.choice(G.n, size=G.n - 37, replace=False)) if subset else None
    nr = G.n if rows is None else rows.size
    c = cov if rows is None else cov[:, rows]
    cz = ((c - c.mean(1, keepdims=True)) / np.where(c.std(1, ddof=1, keepdims=True) > 0,
                                                    c.std(1, ddof=1, keepdims=True), np.inf)).T
    Z = np_Z(codes, rows)
    y = Z[:, [10, 500, 1500]] @ np.array([0.6, -0.5, 0.4]) + cz[:, [0, 2]] @ np.array([1.2, 0.8]) \
        + rng.normal(size=nr)
    fo = oracle.iht(G, y, 8, rows=rows, cov=cov, variant=variant)
    fg = iht.iht_fit_trace(ds, y, 8, rows=rows, variant=variant)
    assert fg.beta.size == G.p + cov.shape[0]
    assert np.any(fo.support >= G.p), "the signal puts covariates in the support"
    got = compare_fits(fo, fg, 8)
    assert got == fo.iterations, f"certified {got} of {fo.iterations}"
    assert np.array_equal(fg.support, fo.support) and rel_err(fg.beta, fo.beta) <= 1e-4
    assert fg.beta[G.p + 3] == 0.0                                  # constant column inert
    ds.set_covariates(None)                                         # removed: plain IHT again
    plain = iht.iht_fit(ds, y, 8, rows=rows, variant=variant)
    fresh = iht.iht_fit(load(iht, ctx, G), y, 8, rows=rows, variant=variant)
    assert plain.beta.size == G.p and np.array_equal(plain.beta, fresh.beta)


def test_covariates_and_htp_limits(iht, ctx):
    rng, G, codes, cov = cov_panel(600, n=300, p=400)
    ds = load(iht, ctx, G)
    y = rng.normal(size=G.n)
    with pytest.raises(iht.IhtError):                     # HTP: single solves only
        iht.iht_fit_batch(ds, [(y, 5, None), (y, 6, None)], variant="htp")
    ds.set_covariates(cov)
    with pytest.raises(iht.IhtError):
        iht.iht_fit_batch(ds, [(y, 5, None), (y, 6, None)])
    with pytest.raises(iht.IhtError):
        iht.iht_cv(ds, y, np.arange(G.n) % 3, [2, 4])
    with pytest.raises(iht.IhtError):
        iht.Server(ds)
    bad = cov.copy()
    bad[1, 17] = np.inf
    ds.set_covariates(bad)
    assert iht.iht_fit(ds, y, 5).status == iht.IHT_ENUMERIC
    with pytest.raises(iht.IhtError):
        ds.set_covariates(np.zeros((65, G.n)))            # more than 64 covariates
