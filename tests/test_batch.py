"""Batched solves and the multi-column gradient against the FP64 oracle (needs a B300).

Bars as for single solves: gradient columns max|dg| / max|g| <= 1e-5; a
solve's support, iteration count and status equal to the oracle's and beta
within 1e-4 whenever the oracle certifies every selection of that solve (the
k-th and (k+1)-th |w| further apart than the FP32 gradient error can move
them, no backtracking test within 1e-3 of its threshold); cross-validated
out-of-fold MSE per model size within 1e-4 of the oracle's.
"""
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


def _torch():
    import torch
    return torch


def load(iht, ctx, G):
    return iht.Dataset(ctx, np.concatenate([MAGIC, G.body]), G.n, G.p)


def rel_err(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def certified(fo):
    tr = fo.trace
    return all(tr["gap"][t] > 10 * GTOL * tr["wscale"][t] and not (tr["margin"][t] < 1e-3)
               for t in range(fo.iterations))


def check_solve(fo, fg):
    """True when the oracle certifies the whole solve (and then it must match)."""
    if not certified(fo):
        return False
    assert fg.iterations == fo.iterations
    assert fg.status == fo.status
    assert np.array_equal(np.asarray(fg.support), fo.support)
    assert rel_err(fg.beta, fo.beta) <= BTOL
    assert abs(fg.objective - fo.objective) <= 1e-6 * fo.objective
    return True


@pytest.mark.parametrize("impl", [1, 2])
@pytest.mark.parametrize("n,p,b", [(37, 5, 1), (1000, 300, 3), (1003, 611, 17), (300, 1000, 5),
                                   (4099, 257, 9), (2000, 1500, 40)])
def test_gradient_batch_parity(iht, ctx, impl, n, p, b):
    torch = _torch()
    rng = np.random.default_rng(11 * n + p + b)
    G, _ = random_geno(rng, n, p, miss=0.02)
    ds = load(iht, ctx, G)
    sets = [None, np.sort(rng.choice(n, size=n - n // 5, replace=False)).astype(np.int32),
            np.sort(rng.choice(n, size=max(1, n // 2), replace=False)).astype(np.int32)]
    rows = [sets[c % 3] for c in range(b)]
    R = [rng.normal(size=n if r is None else r.size).astype(np.float32) * (1 + c)
         for c, r in enumerate(rows)]
    dev_rows = {id(r): torch.from_numpy(r).cuda() for r in sets if r is not None}
    Gd = iht.iht_gradient_batch(ds, [torch.from_numpy(r).cuda() for r in R],
                                [None if r is None else dev_rows[id(r)] for r in rows],
                                impl=impl).cpu().numpy()
    for c in range(b):
        go = oracle.gradient(G, R[c].astype(np.float64), rows[c])
        assert rel_err(Gd[c], go) <= GTOL, f"column {c}"


def test_gradient_batch_two_passes(iht, ctx):
    """More columns than one pass holds (44): the passes split and agree."""
    torch = _torch()
    rng = np.random.default_rng(77)
    n, p, b = 700, 900, 130
    G, _ = random_geno(rng, n, p, miss=0.02)
    ds = load(iht, ctx, G)
    R = rng.normal(size=(b, n)).astype(np.float32)
    Gd = iht.iht_gradient_batch(ds, [torch.from_numpy(R[c]).cuda() for c in range(b)],
                                impl=2).cpu().numpy()
    for c in (0, 1, 43, 44, 57, 87, 88, 111, 112, 129):
        assert rel_err(Gd[c], oracle.gradient(G, R[c].astype(np.float64))) <= GTOL


def test_gradient_batch_matches_single_column(iht, ctx):
    """One column of the multi-column pass against the same column alone: the
    passes share the limb representation, the K order and the rounding of every
    step, so the column is bit-identical to the single-column pass."""
    torch = _torch()
    rng = np.random.default_rng(5)
    G, _ = random_geno(rng, 1500, 700, miss=0.02)
    ds = load(iht, ctx, G)
    r = rng.normal(size=1500).astype(np.float32)
    g1 = iht.iht_gradient(ds, torch.from_numpy(r).cuda(), impl=1).cpu().numpy()
    g2 = iht.iht_gradient(ds, torch.from_numpy(r).cuda(), impl=2).cpu().numpy()
    others = [torch.from_numpy(rng.normal(size=1500).astype(np.float32)).cuda() for _ in range(20)]
    gb = iht.iht_gradient_batch(ds, others[:7] + [torch.from_numpy(r).cuda()] + others[7:],
                                impl=2).cpu().numpy()
    assert rel_err(gb[7], g1) <= GTOL
    assert np.array_equal(gb[7], g2)


def _signal_panel(seed, n, p, k_star, effect=0.6, miss=0.02):
    rng = np.random.default_rng(seed)
    G, codes = random_geno(rng, n, p, miss=miss)
    Z = np_Z(codes)
    causal = np.sort(rng.choice(p, size=k_star, replace=False))
    y = Z[:, causal] @ (rng.choice([-1, 1], size=k_star) * effect) + rng.normal(size=n)
    return G, codes, y, causal, rng


@pytest.mark.parametrize("impl", [1, 2])
def test_fit_batch_cv_against_oracle(iht, ctx, impl):
    """5-fold cross-validation over k in {2, 4, 6}: every certified solve
    equals the oracle's, and the out-of-fold MSE curve matches."""
    torch = _torch()
    n, p, folds, ks = 640, 1800, 5, (2, 4, 6)
    G, codes, y, causal, rng = _signal_panel(3, n, p, 4)
    ds = load(iht, ctx, G)
    lab = synth.cv_folds(n, folds, 9)
    train = [np.flatnonzero(lab != f).astype(np.int32) for f in range(folds)]
    test = [np.flatnonzero(lab == f).astype(np.int32) for f in range(folds)]
    probs = [(y[train[f]], k, train[f]) for f in range(folds) for k in ks]
    res = iht.iht_fit_batch(ds, probs, grad_impl=impl)
    ncert = 0
    mse_g = np.zeros(len(ks))
    mse_o = np.zeros(len(ks))
    for i, (f, k) in enumerate([(f, k) for f in range(folds) for k in ks]):
        fo = oracle.iht(G, y[train[f]], k, rows=train[f])
        ncert += check_solve(fo, res[i])
        assert np.count_nonzero(res[i].beta) <= k
        _, ut, vt = oracle.counts(G, train[f])
        for beta, acc in ((res[i].beta, mse_g), (fo.beta, mse_o)):
            cols = np.flatnonzero(beta).astype(np.int32)
            pred = oracle.zmul(G, cols, beta[cols], test[f], ut, vt) if cols.size else 0.0
            acc[ks.index(k)] += np.mean((y[test[f]] - pred) ** 2) / folds
    print(f"[parity] CV batch: {ncert} of {len(probs)} certified, tie-ambiguous "
          f"exclusion {1 - ncert / len(probs):.3f}")
    assert ncert == len(probs)                         # every solve certified: all must match
    assert np.max(np.abs(mse_g - mse_o) / mse_o) <= BTOL
    assert ks[int(np.argmin(mse_g))] == ks[int(np.argmin(mse_o))]


def test_fit_batch_mixed_sizes_and_sets(iht, ctx):
    """Different k, row sets and phenotypes in one batch; each against the oracle."""
    n, p = 900, 2500
    G, codes, y0, _, rng = _signal_panel(8, n, p, 6, effect=0.5)
    ds = load(iht, ctx, G)
    sub = np.sort(rng.choice(n, size=700, replace=False)).astype(np.int32)
    Z = np_Z(codes)
    y1 = Z[:, [5, 77, 900]] @ np.array([0.7, -0.6, 0.8]) + rng.normal(size=n)
    probs = [(y0, 6, None), (y1, 3, None), (y0[sub], 9, sub), (y1[sub], 1, sub),
             (y0, 25, None), (y1, 12, None)]
    res = iht.iht_fit_batch(ds, probs, grad_impl=2)
    ncert = 0
    for (yy, k, rows), fg in zip(probs, res):
        fo = oracle.iht(G, yy, k, rows=rows)
        ncert += check_solve(fo, fg)
        assert np.count_nonzero(fg.beta) <= k and len(fg.support) == k
    print(f"[parity] mixed batch: {ncert} of {len(probs)} certified")
    assert ncert == len(probs)


def test_fit_batch_status_and_io(iht, ctx):
    torch = _torch()
    rng = np.random.default_rng(21)
    G, _ = random_geno(rng, 400, 300, miss=0.02)
    ds = load(iht, ctx, G)
    y = rng.normal(size=400)
    bad = y.copy()
    bad[3] = np.inf
    res = iht.iht_fit_batch(ds, [(y, 5, None), (bad, 5, None), (np.zeros(400), 3, None), (y, 8, None)])
    assert res[1].status == iht.IHT_ENUMERIC and res[1].iterations == 0
    assert res[2].status == iht.IHT_OK and res[2].iterations == 0 and not res[2].beta.any()
    assert res[0].iterations > 0 and res[3].iterations > 0
    # the good solves are unaffected by their neighbours
    alone = iht.iht_fit_batch(ds, [(y, 5, None)])[0]
    if certified(oracle.iht(G, y, 5)):
        assert np.array_equal(alone.support, res[0].support)
        assert alone.iterations == res[0].iterations
        assert rel_err(alone.beta, res[0].beta) <= BTOL
    with pytest.raises(iht.IhtError):
        iht.iht_fit_batch(ds, [(y[:3], 2, np.array([1, 1, 2], np.int32))])    # duplicate row
    with pytest.raises(iht.IhtError):
        iht.iht_fit_batch(ds, [(y, 301, None)])                                # k > p
    with pytest.raises(iht.IhtError):
        iht.iht_fit_batch(ds, [(y[:1], 1, np.array([4], np.int32))])           # n_rows < 2
    # device inputs and outputs give the host results bit for bit; runs repeat exactly
    a = iht.iht_fit_batch(ds, [(y, 5, None), (y, 8, None)])
    yd = torch.from_numpy(y).cuda()
    b = iht.iht_fit_batch(ds, [(yd, 5, None), (yd, 8, None)], out_device=True)
    c = iht.iht_fit_batch(ds, [(y, 5, None), (y, 8, None)])
    d = iht.iht_fit_batch(ds, [(yd, 5, None), (yd, 8, None)], out_device=True, dense=False)
    for i in range(2):
        assert np.array_equal(a[i].beta, b[i].beta.cpu().numpy())
        assert np.array_equal(a[i].support, b[i].support.cpu().numpy())
        assert np.array_equal(a[i].beta, c[i].beta)
        assert np.array_equal(a[i].beta[a[i].support], a[i].beta_s)
        assert d[i].beta is None
        assert np.array_equal(d[i].support.cpu().numpy(), a[i].support)
        assert np.array_equal(d[i].beta_s.cpu().numpy(), a[i].beta_s)


def test_fit_batch_matches_single_solves(iht, ctx):
    """A solve in a batch and the same solve alone through iht_fit: the same
    arithmetic step for step, so the same support, beta bit for bit and the
    same iteration count, whatever else is in the batch."""
    n, p = 1200, 3001
    G, codes, y, _, rng = _signal_panel(12, n, p, 5, effect=0.5)
    ds = load(iht, ctx, G)
    rows = np.sort(rng.choice(n, size=1000, replace=False)).astype(np.int32)
    y2 = rng.normal(size=n)
    probs = [(y, 5, None), (y[rows], 5, rows), (y, 10, None), (y2, 3, None), (y2[rows], 40, rows)]
    res = iht.iht_fit_batch(ds, probs)
    for (yy, k, rr), fb in zip(probs, res):
        fs = iht.iht_fit(ds, yy, k, rows=rr)
        assert np.array_equal(fs.support, fb.support)
        assert np.array_equal(fs.beta, fb.beta)
        assert fs.iterations == fb.iterations and fs.status == fb.status
        assert fs.objective == fb.objective


def test_fit_batch_iteration_graphs(iht, ctx):
    """An iteration replays a cached CUDA graph of the same launches in the same
    order (gradient pass, selection, step, two attempts) once a graph for its
    number of active columns exists, so a batch gives the same bits on its
    first call, on a repeat that replays the cached graphs from its second
    iteration on, alone (a one-column batch runs the single-column pass inside
    its graph) and through iht_fit."""
    n, p = 1200, 3001
    G, codes, y, _, rng = _signal_panel(12, n, p, 5, effect=0.5)
    ds = load(iht, ctx, G)
    y2 = rng.normal(size=n)
    probs = [(y, 5, None), (y2, 3, None), (y, 10, None)]
    first = iht.iht_fit_batch(ds, probs)
    again = iht.iht_fit_batch(ds, probs)
    assert first[0].graph_replays > 0
    its = max(r.iterations for r in first)
    assert first[0].graph_replays <= again[0].graph_replays <= its - 1
    for (yy, k, rr), f, a in zip(probs, first, again):
        one = iht.iht_fit_batch(ds, [(yy, k, rr)])[0]
        s = iht.iht_fit(ds, yy, k, rows=rr)
        assert f.iterations > 2 and one.graph_replays > 0 and s.graph_replays > 0
        for r in (a, one, s):
            assert np.array_equal(r.support, f.support) and np.array_equal(r.beta, f.beta)
            assert (r.iterations, r.status, r.objective) == (f.iterations, f.status, f.objective)
    # profiled: every gradient pass, direct or replayed, is timed (one per iteration)
    pr = iht.iht_fit_batch(ds, probs, profile=1)
    its = max(r.iterations for r in pr)
    assert its - 1 <= pr[0].grad_launches <= its + 1 and pr[0].grad_ms > 0
    assert all(np.array_equal(r.beta, f.beta) for r, f in zip(pr, first))


def test_fit_batch_odd_p(iht, ctx):
    """p not a multiple of 4: per-solve gradient rows start off 16-byte boundaries."""
    n, p = 500, 1003
    G, codes, y, _, rng = _signal_panel(31, n, p, 3, effect=0.7)
    ds = load(iht, ctx, G)
    probs = [(y, 3, None), (y, 5, None), (y, 2, None)]
    res = iht.iht_fit_batch(ds, probs)
    for (yy, k, rows), fg in zip(probs, res):
        check_solve(oracle.iht(G, yy, k, rows=rows), fg)
        s = iht.iht_fit(ds, yy, k, rows=rows)
        if certified(oracle.iht(G, yy, k, rows=rows)):
            assert np.array_equal(s.support, fg.support)


@pytest.mark.parametrize("cfg,b", [(3, 44), (4, 64), (5, 32)])
def test_fullsize_gradient_batch_sampled(iht, ctx, cfg, b):
    """The full panels of the batched workloads (CV n=6000 p=1M, serving n=10000
    p=1M, large n=20000 p=4M) in the multi-column launch shape their loops use
    (one 44-column pass over the five training folds; 64 request-sized subsets,
    two passes; 32 phenotypes on all rows): every column on sampled SNPs against
    the oracle."""
    torch = _torch()
    pn = synth.config_panel(cfg)
    bed = pn.bed()
    ds = iht.Dataset(ctx, bed, pn.n, pn.p)
    rng = np.random.default_rng(100 + cfg)
    if cfg == 3:
        lab = synth.cv_folds(pn.n, 5, 7)
        sets = [np.flatnonzero(lab != f).astype(np.int32) for f in range(5)]
    elif cfg == 4:
        sets = [np.sort(rng.choice(pn.n, size=int(rng.integers(2000, pn.n + 1)), replace=False))
                .astype(np.int32) for _ in range(8)]
    else:
        sets = [None]
    rows = [sets[c % len(sets)] for c in range(b)]
    R = [rng.normal(size=pn.n if r is None else r.size).astype(np.float32) for r in rows]
    dev_rows = {id(r): torch.from_numpy(r).cuda() for r in sets if r is not None}
    Gd = iht.iht_gradient_batch(ds, [torch.from_numpy(x).cuda() for x in R],
                                [None if r is None else dev_rows[id(r)] for r in rows])
    snps = np.sort(rng.choice(pn.p, size=1500, replace=False))
    Gs = oracle.Geno(bed[3:].reshape(pn.p, pn.bed_row_bytes)[snps].ravel(), pn.n, snps.size,
                     pn.bed_row_bytes)
    Gh = Gd[:, torch.from_numpy(snps).cuda()].cpu().numpy()
    for c in range(b):
        go = oracle.gradient(Gs, R[c].astype(np.float64), rows[c])
        assert rel_err(Gh[c], go) <= GTOL, f"column {c}"
    assert bool(torch.isfinite(Gd).all())
    del Gd, ds, bed
