"""CUDA path against the FP64 oracle, through the C ABI (needs a B300).

Bars: integer work (decode, counts, supports) bit-exact; FP64 statistics
bit-exact (same correctly rounded expression); gradient max|dg| / max|g| <= 1e-5;
beta max|db| / max|b| <= 1e-4; supports compared where the oracle certifies that
the k-th and (k+1)-th |w| are further apart than the FP32 gradient error can
move them and no backtracking decision sits within 1e-3 of its threshold.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from pins import np_Z, random_geno

pytestmark = pytest.mark.gpu

GTOL = 1e-5
BTOL = 1e-4
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


def load(iht, ctx, G: oracle.Geno):
    assert G.row_bytes == (G.n + 3) // 4
    return iht.Dataset(ctx, np.concatenate([MAGIC, G.body]), G.n, G.p)


def rel_err(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


SHAPES = [(1, 3), (2, 5), (3, 7), (5, 1), (13, 40), (64, 33), (1000, 300), (1001, 129),
          (1002, 77), (1003, 65)]


@pytest.mark.parametrize("n,p", SHAPES)
def test_counts_bit_exact(iht, ctx, n, p):
    rng = np.random.default_rng(n * 1000 + p)
    G, _ = random_geno(rng, n, p, miss=0.05)
    ds = load(iht, ctx, G)
    rowsets = [None]
    if n >= 4:
        rowsets.append(np.sort(rng.choice(n, size=n // 2, replace=False)).astype(np.int32))
    for rows in rowsets:
        c, u, v = iht.iht_counts(ds, rows)
        co, uo, vo = oracle.counts(G, rows)
        assert np.array_equal(c, co)
        assert np.array_equal(u, uo) and np.array_equal(v, vo)


def _torch():
    import torch
    return torch


@pytest.mark.parametrize("impl", [0, 1, 2])
@pytest.mark.parametrize("n,p", [(1, 3), (37, 5), (1000, 300), (1003, 611), (4099, 257), (300, 1000)])
def test_gradient_parity(iht, ctx, impl, n, p):
    torch = _torch()
    rng = np.random.default_rng(7 + n + p)
    G, _ = random_geno(rng, n, p, miss=0.02)
    ds = load(iht, ctx, G)
    for rows in (None, np.sort(rng.choice(n, size=n - n // 3, replace=False)).astype(np.int32)):
        nr = n if rows is None else rows.size
        r = rng.normal(size=nr).astype(np.float32)
        g = iht.iht_gradient(ds, torch.from_numpy(r).cuda(), None if rows is None else
                             torch.from_numpy(rows).cuda(), impl=impl).cpu().numpy()
        go = oracle.gradient(G, r.astype(np.float64), rows)
        assert rel_err(g, go) <= GTOL


@pytest.mark.parametrize("n", [40500, 41000])
def test_gradient_long_residual_paths(iht, ctx, n):
    """Sample counts past the interleaved missing-call lists: n_pad = 40 960 sums
    over the plain lists with r in shared memory, n = 41 000 over the global-
    memory kernel (r too long for shared memory); gradient and a short solve
    against the oracle."""
    torch = _torch()
    rng = np.random.default_rng(n)
    G, codes = random_geno(rng, n, 40, miss=0.02)
    ds = load(iht, ctx, G)
    r = rng.normal(size=n).astype(np.float32)
    g = iht.iht_gradient(ds, torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel_err(g, oracle.gradient(G, r.astype(np.float64))) <= GTOL
    Z = np_Z(codes)
    y = Z[:, [3, 17, 29]] @ np.array([0.4, -0.3, 0.5]) + rng.normal(size=n)
    fg = iht.iht_fit(ds, y, 3)
    fo = oracle.iht(G, y, 3, trace=False)
    assert np.array_equal(np.asarray(fg.support), np.asarray(fo.support))
    assert fg.status == fo.status


def test_gradient_uncentred_residual(iht, ctx):
    """A residual with a large mean: the R and M terms still cancel correctly."""
    torch = _torch()
    rng = np.random.default_rng(3)
    G, _ = random_geno(rng, 2000, 400, miss=0.02)
    ds = load(iht, ctx, G)
    r = (rng.normal(size=2000) + 0.3).astype(np.float32)
    g = iht.iht_gradient(ds, torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel_err(g, oracle.gradient(G, r.astype(np.float64))) <= GTOL


@pytest.mark.parametrize("p,k", [(1, 1), (10, 3), (1000, 7), (100003, 100), (4096 * 3 + 5, 2048)])
@pytest.mark.parametrize("kind", ["real", "ties", "sparse"])
def test_topk_matches_lexsort(iht, ctx, p, k, kind):
    torch = _torch()
    rng = np.random.default_rng(p + k)
    if kind == "real":
        w = rng.normal(size=p).astype(np.float32)
    elif kind == "ties":
        w = rng.integers(-3, 4, size=p).astype(np.float32)
    else:
        w = np.zeros(p, np.float32)
        nz = rng.choice(p, size=max(1, p // 50), replace=False)
        w[nz] = rng.normal(size=nz.size)
    idx = iht.iht_topk(ctx, torch.from_numpy(w).cuda(), k).cpu().numpy()
    want = np.sort(np.lexsort((np.arange(p), -np.abs(w.astype(np.float64))))[:k])
    assert np.array_equal(idx, want)


def test_zmul_parity(iht, ctx):
    torch = _torch()
    rng = np.random.default_rng(9)
    G, _ = random_geno(rng, 777, 500, miss=0.03)
    ds = load(iht, ctx, G)
    cols = rng.choice(500, size=40, replace=False).astype(np.int32)
    coef = rng.normal(size=40)
    rows = np.sort(rng.choice(777, size=500, replace=False)).astype(np.int32)
    out = iht.iht_zmul(ds, torch.from_numpy(cols).cuda(), torch.from_numpy(coef).cuda(),
                       rows=torch.from_numpy(rows).cuda()).cpu().numpy()
    want = oracle.zmul(G, cols, coef, rows)
    assert rel_err(out, want) <= 1e-12
    # held-out rows standardised with another row set's statistics
    _, ut, vt = oracle.counts(G, np.arange(0, 777, 2))
    te = np.arange(1, 777, 2).astype(np.int32)
    out = iht.iht_zmul(ds, torch.from_numpy(cols).cuda(), torch.from_numpy(coef).cuda(),
                       rows=torch.from_numpy(te).cuda(), u=torch.from_numpy(ut).cuda(),
                       v=torch.from_numpy(vt).cuda()).cpu().numpy()
    assert rel_err(out, oracle.zmul(G, cols, coef, te, ut, vt)) <= 1e-12


def lead_certified(fo):
    """Iterations the oracle certifies before its first tie-ambiguous one."""
    tr = fo.trace
    for t in range(fo.iterations):
        if not (tr["gap"][t] > 10 * GTOL * tr["wscale"][t] and not (tr["margin"][t] < 1e-3)):
            return t
    return fo.iterations


def report_exclusion(name, certified, total):
    """Prints the tie-ambiguous exclusion rate: iterations (or solves) the
    oracle does not certify, which the comparison leaves out."""
    rate = 1.0 - certified / max(total, 1)
    print(f"[parity] {name}: {certified} of {total} certified, tie-ambiguous exclusion {rate:.3f}")
    return rate


def compare_fits(fo, fg, k):
    """Per-iteration comparison while the oracle certifies the selections."""
    T = min(fo.iterations, fg.iterations)
    certified = 0
    for t in range(T):
        tr = fo.trace
        ok = tr["gap"][t] > 10 * GTOL * tr["wscale"][t] and not (tr["margin"][t] < 1e-3)
        if not ok:
            break
        assert np.array_equal(fg.trace["supp"][t], tr["supp"][t]), f"support at iteration {t}"
        assert rel_err(fg.trace["beta"][t], tr["beta"][t]) <= BTOL, f"beta at iteration {t}"
        assert fg.trace["backtracks"][t] == tr["backtracks"][t]
        assert abs(fg.trace["objective"][t] - tr["objective"][t]) <= 1e-6 * tr["objective"][t]
        certified += 1
    if certified == T and fo.iterations == fg.iterations:
        assert np.array_equal(fg.support, fo.support)
        assert rel_err(fg.beta, fo.beta) <= BTOL
        assert fg.status == fo.status
    return certified


def test_fit_parity_config1(iht, ctx):
    pn = synth.config_panel(1)
    G = oracle.Geno.from_bed(pn.bed(), pn.n, pn.p)
    ds = load(iht, ctx, G)
    y, causal, _ = synth.config_phenotype(1, pn)
    fo = oracle.iht(G, y, 10)
    assert report_exclusion("config 1", lead_certified(fo), fo.iterations) == 0.0
    for impl in (1, 2):
        fg = iht.iht_fit_trace(ds, y, 10, grad_impl=impl)
        assert compare_fits(fo, fg, 10) == fo.iterations
        assert np.count_nonzero(fg.beta) <= 10
        obj = np.concatenate([[0.5 * y @ y], fg.trace["objective"]])
        assert np.all(np.diff(obj) <= 1e-9 * obj[:-1])


@pytest.mark.parametrize("seed", range(6))
def test_fit_parity_small_panels(iht, ctx, seed):
    rng = np.random.default_rng(100 + seed)
    n = [150, 333, 401, 64, 1000, 257][seed]
    p = [80, 500, 1201, 40, 3000, 9][seed]
    k = [5, 12, 30, 1, 20, 9][seed]
    G, codes = random_geno(rng, n, p, miss=0.02)
    ds = load(iht, ctx, G)
    rows = None if seed % 2 == 0 else np.sort(rng.choice(n, size=n - 11, replace=False))
    nr = n if rows is None else rows.size
    # a sparse signal plus noise (and an offset: the solver must not need centred y)
    Z = np_Z(codes, rows)
    causal = rng.choice(p, size=min(k, p), replace=False)
    y = Z[:, causal] @ rng.normal(0, 0.5, size=causal.size) + rng.normal(size=nr) + 0.5
    fo = oracle.iht(G, y, k, rows=rows, max_iter=60, tol=1e-6)
    fg = iht.iht_fit_trace(ds, y, k, rows=rows, max_iter=60, tol=1e-6)
    # the oracle certifies every iteration of these seeds; each must agree, and
    # the GPU solve must take the same number of iterations to the same result
    assert report_exclusion(f"small panel {seed}", lead_certified(fo), fo.iterations) == 0.0
    assert compare_fits(fo, fg, k) == fo.iterations == fg.iterations
    obj = np.concatenate([[0.5 * y @ y], fg.trace["objective"]])
    assert np.all(np.diff(obj) <= 1e-9 * obj[:-1])


def test_fit_k_equals_p_is_ols(iht, ctx):
    rng = np.random.default_rng(41)
    G, codes = random_geno(rng, 120, 6, miss=0.0)
    ds = load(iht, ctx, G)
    Z = np_Z(codes)
    y = Z @ rng.normal(size=6) + rng.normal(size=120)
    fg = iht.iht_fit(ds, y, 6, tol=1e-10, max_iter=20000)
    coef, *_ = np.linalg.lstsq(Z, y, rcond=None)
    assert rel_err(fg.beta, coef) <= 1e-5


def test_fit_status_and_io_paths(iht, ctx):
    torch = _torch()
    rng = np.random.default_rng(5)
    G, _ = random_geno(rng, 300, 200, miss=0.02)
    ds = load(iht, ctx, G)
    y = rng.normal(size=300)
    bad = y.copy()
    bad[17] = np.nan
    assert iht.iht_fit(ds, bad, 5).status == iht.IHT_ENUMERIC
    with pytest.raises(iht.IhtError):
        iht.iht_fit(ds, y[:1], 5, rows=np.array([3], np.int32))          # n_rows < 2
    with pytest.raises(iht.IhtError):
        iht.iht_fit(ds, y[:3], 5, rows=np.array([3, 3, 4], np.int32))    # duplicate row
    with pytest.raises(iht.IhtError):
        iht.iht_fit(ds, y, 201)                                           # k > p
    z = iht.iht_fit(ds, np.zeros(300), 4)
    assert z.status == iht.IHT_OK and z.iterations == 0 and not z.beta.any()
    a = iht.iht_fit(ds, y, 7)
    b = iht.iht_fit(ds, torch.from_numpy(y).cuda(), 7, out_device=True)
    assert np.array_equal(a.beta, b.beta.cpu().numpy())
    assert np.array_equal(a.support, b.support.cpu().numpy())
    c = iht.iht_fit(ds, y, 7)
    assert np.array_equal(a.beta, c.beta) and a.iterations == c.iterations   # run to run
    # the zeroed-output flag: the binding passes calloc'ed zeros and sets it;
    # without it the library zero-fills a dirty buffer itself; other bits: EINVAL
    o = iht.iht_default_options()
    beta = np.full(ds.p, 7.0)
    supp = np.empty(7, np.int32)
    res = iht.iht_result()
    yy = np.ascontiguousarray(y, dtype=np.float64)
    rc = iht._lib().iht_fit(ds.h, None, ds.n, ctypes.c_void_p(yy.ctypes.data), 7, ctypes.byref(o),
                            ctypes.c_void_p(beta.ctypes.data), ctypes.c_void_p(supp.ctypes.data),
                            ctypes.byref(res))
    assert rc == a.status and np.array_equal(beta, a.beta) and np.array_equal(supp, a.support)
    o.flags = 2
    assert iht._lib().iht_fit(ds.h, None, ds.n, ctypes.c_void_p(yy.ctypes.data), 7, ctypes.byref(o),
                              ctypes.c_void_p(beta.ctypes.data), ctypes.c_void_p(supp.ctypes.data),
                              ctypes.byref(res)) == iht.IHT_EINVAL


@pytest.fixture(scope="module")
def cfg2(iht, ctx):
    pn = synth.config_panel(2)
    bed = pn.bed()
    ds = iht.Dataset(ctx, bed, pn.n, pn.p)
    return pn, bed, ds


def test_fullsize_gradient_sampled(iht, cfg2):
    """n=5000, p=500000 (the single-solve bench workload): sampled SNPs against the oracle."""
    torch = _torch()
    pn, bed, ds = cfg2
    rng = np.random.default_rng(2)
    r = rng.normal(size=pn.n).astype(np.float32)
    snps = np.sort(rng.choice(pn.p, size=3000, replace=False))
    rb = pn.bed_row_bytes
    body = bed[3:].reshape(pn.p, rb)[snps].ravel()
    Gs = oracle.Geno(body, pn.n, snps.size, rb)
    go = oracle.gradient(Gs, r.astype(np.float64))
    for impl in (1, 2):
        g = iht.iht_gradient(ds, torch.from_numpy(r).cuda(), impl=impl).cpu().numpy()
        assert rel_err(g[snps], go) <= GTOL
    # the full gradient is finite and no SNP is skipped
    assert np.all(np.isfinite(g)) and np.count_nonzero(g) > 0.99 * pn.p


def test_fullsize_fit(iht, cfg2):
    """Full single-solve workload against the oracle (same supports, beta within 1e-4)."""
    pn, bed, ds = cfg2
    y, causal, _ = synth.config_phenotype(2, pn)
    fg = iht.iht_fit_trace(ds, y, 50)
    G = oracle.Geno.from_bed(bed, pn.n, pn.p)
    fo = oracle.iht(G, y, 50)
    # all 16 iterations (15 shrinks) are certified: each one, the final support,
    # beta and status must agree
    assert report_exclusion("n=5000 p=500000 k=50", lead_certified(fo), fo.iterations) == 0.0
    assert compare_fits(fo, fg, 50) == fo.iterations == fg.iterations
    assert np.array_equal(fg.support, fo.support) and fg.status == fo.status
    assert rel_err(fg.beta, fo.beta) <= BTOL
    plain = iht.iht_fit(ds, y, 50)                     # graph path: the traced path's bits
    assert np.array_equal(plain.beta, fg.beta) and plain.iterations == fg.iterations
    assert np.count_nonzero(fg.beta) <= 50


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_topk_unaligned_keys(iht, ctx, offset):
    """Keys that do not start on a 16-byte boundary (a slice of a larger array)."""
    torch = _torch()
    rng = np.random.default_rng(offset)
    p, k = 50003, 37
    w = rng.normal(size=p + offset).astype(np.float32)
    wd = torch.from_numpy(w).cuda()[offset:]
    idx = iht.iht_topk(ctx, wd, k).cpu().numpy()
    ww = w[offset:].astype(np.float64)
    assert np.array_equal(idx, np.sort(np.lexsort((np.arange(p), -np.abs(ww)))[:k]))


def test_topk_nan_is_reported(iht, ctx):
    """A NaN key: iht_topk reports ENUMERIC; the next clean call is OK again."""
    torch = _torch()
    rng = np.random.default_rng(12)
    w = rng.normal(size=20000).astype(np.float32)
    bad = w.copy()
    bad[777] = np.nan
    with pytest.raises(iht.IhtError) as e:
        iht.iht_topk(ctx, torch.from_numpy(bad).cuda(), 10)
    assert e.value.status == iht.IHT_ENUMERIC
    idx = iht.iht_topk(ctx, torch.from_numpy(w).cuda(), 10).cpu().numpy()
    assert np.array_equal(idx, np.sort(np.lexsort((np.arange(w.size), -np.abs(w.astype(np.float64))))[:10]))


@pytest.mark.parametrize("case", ["config1", "rows", "covariates", "k256", "backtracking"])
def test_fused_solve_matches_per_iteration_paths(iht, ctx, case):
    """A solve run as one graph (the fused per-iteration kernel in a conditional
    loop) gives the bits of the per-iteration graph (profiled solves) and of the
    traced per-launch path, and launches a few kernels per iteration."""
    rng = np.random.default_rng(55)
    if case == "config1":
        pn = synth.config_panel(1)
        G = oracle.Geno.from_bed(pn.bed(), pn.n, pn.p)
        y, _, _ = synth.config_phenotype(1, pn)
        rows, k, kw = None, 10, {}
    else:
        G, codes = random_geno(rng, 700, 3000, miss=0.02)
        Z = np_Z(codes)
        y = Z[:, rng.choice(3000, 12, replace=False)] @ rng.normal(0, 0.5, 12) + rng.normal(size=700)
        rows, k, kw = None, 12, {}
        if case == "rows":
            rows = np.sort(rng.choice(700, size=611, replace=False)).astype(np.int32)
            y = y[rows]
        if case == "k256":
            k = 256
        if case == "backtracking":
            kw = dict(c=0.3)
    ds = load(iht, ctx, G)
    if case == "covariates":
        ds.set_covariates(np.vstack([rng.normal(size=G.n), rng.gamma(2.0, size=G.n)]))
    l0 = iht.iht_kernel_launches()
    a = iht.iht_fit(ds, y, k, rows=rows, **kw)
    launches = iht.iht_kernel_launches() - l0
    b = iht.iht_fit(ds, y, k, rows=rows, profile=1, **kw)
    c = iht.iht_fit_trace(ds, y, k, rows=rows, **kw)
    for other in (b, c):
        assert np.array_equal(a.beta, other.beta) and np.array_equal(a.support, other.support)
        assert (a.iterations, a.status, a.backtracks) == (other.iterations, other.status, other.backtracks)
        assert a.objective == other.objective and a.mu == other.mu
    print(f"[fused] {case}: {a.iterations} iterations, {a.backtracks} shrinks, {launches} launches")
    assert a.iterations >= 2 and launches <= 12 + 6 * a.iterations
    if case == "backtracking":
        assert a.backtracks > 0
