"""Model selection by q-fold cross-validation and refit (Sec. 2.4) against the oracle.

Bars: the averaged out-of-fold MSE curve within 1e-4 relative of the oracle's
and the same k_best; the refit's support, iterations and beta as for single
solves whenever the oracle certifies it; and, independent of how close the
fits are, the device's MSE of its own fold fits equal to the FP64 MSE of those
fits (the oracle's product with the training rows' statistics) to 1e-12.
Argument checks run on the host.
"""
import numpy as np
import pytest

import oracle
import paper_1608_01398_b300 as iht
import synth
from pins import np_Z, random_geno

BTOL = 1e-4
GTOL = 1e-5
MAGIC = np.array([0x6C, 0x1B, 0x01], dtype=np.uint8)


def test_cv_arguments_on_the_host():
    L = iht._lib()
    ks = np.array([1, 2], np.int32)
    fold = np.zeros(4, np.int32)
    y = np.zeros(4)
    assert L.iht_cv(None, y.ctypes.data, fold.ctypes.data, 2, ks.ctypes.data, 2, None, None, None,
                    None, None, None, None) == iht.IHT_EINVAL


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return iht.Context(0)


def _panel(seed, n, p, k_star, effect=0.6, miss=0.02):
    rng = np.random.default_rng(seed)
    G, codes = random_geno(rng, n, p, miss=miss)
    Z = np_Z(codes)
    causal = np.sort(rng.choice(p, size=k_star, replace=False))
    y = Z[:, causal] @ (rng.choice([-1, 1], size=k_star) * effect) + rng.normal(size=n)
    return G, y, rng


def _load(ctx, G):
    return iht.Dataset(ctx, np.concatenate([MAGIC, G.body]), G.n, G.p)


def _certified(fo):
    tr = fo.trace
    return all(tr["gap"][t] > 10 * GTOL * tr["wscale"][t] and not (tr["margin"][t] < 1e-3)
               for t in range(fo.iterations))


@pytest.mark.gpu
def test_cv_against_oracle(ctx):
    n, p, q, ks = 640, 1800, 5, (2, 4, 6)
    G, y, rng = _panel(3, n, p, 4)
    ds = _load(ctx, G)
    fold = synth.cv_folds(n, q, 9)
    res = iht.iht_cv(ds, y, fold, ks)
    ref = oracle.cv(G, y, fold, q, ks)
    assert np.max(np.abs(res.mse - ref.mse) / ref.mse) <= BTOL
    assert res.mse_fold.shape == (q, len(ks))
    assert np.allclose(res.mse, res.mse_fold.mean(axis=0), rtol=1e-15, atol=0)
    assert res.k_best == ref.k_best
    fo = oracle.iht(G, y, res.k_best)
    if _certified(fo):
        assert np.array_equal(np.asarray(res.fit.support), fo.support)
        assert res.fit.iterations == fo.iterations
        assert np.max(np.abs(res.fit.beta - fo.beta)) <= BTOL * np.max(np.abs(fo.beta))
    # the refit is iht_fit at k_best, bit for bit
    alone = iht.iht_fit(ds, y, res.k_best)
    assert np.array_equal(alone.beta, res.fit.beta) and alone.iterations == res.fit.iterations


@pytest.mark.gpu
def test_cv_mse_of_its_own_fits(ctx):
    """Unequal partitions, 40 held-out subjects (label -1), k = 1 and a size
    above the signal: the device MSE of every (partition, size) fit against the
    FP64 MSE of the same fits, which a batch of the same solves reproduces bit
    for bit; the refit is iht_fit on the labelled rows."""
    n, p, q, ks = 540, 1203, 3, (1, 3, 8)
    G, y, rng = _panel(17, n, p, 3)
    ds = _load(ctx, G)
    fold = rng.permutation(np.repeat(np.arange(-1, q), [40, 120, 170, 210])).astype(np.int32)
    res = iht.iht_cv(ds, y, fold, ks)
    train = [np.flatnonzero((fold != f) & (fold >= 0)).astype(np.int32) for f in range(q)]
    test = [np.flatnonzero(fold == f).astype(np.int32) for f in range(q)]
    fits = iht.iht_fit_batch(ds, [(y[train[f]], k, train[f]) for f in range(q) for k in ks])
    want = np.zeros((q, len(ks)))
    for f in range(q):
        _, ut, vt = oracle.counts(G, train[f])
        for t in range(len(ks)):
            fb = fits[f * len(ks) + t]
            cols = np.asarray(fb.support, dtype=np.int32)
            pred = oracle.zmul(G, cols, fb.beta[cols], test[f], ut, vt)
            want[f, t] = np.mean((y[test[f]] - pred) ** 2)
    assert np.allclose(res.mse_fold, want, rtol=1e-12, atol=0)
    assert res.k_best == ks[int(np.argmin(want.mean(axis=0)))]
    inside = np.flatnonzero(fold >= 0).astype(np.int32)
    alone = iht.iht_fit(ds, y[inside], res.k_best, rows=inside)
    assert np.array_equal(alone.beta, res.fit.beta) and alone.iterations == res.fit.iterations


@pytest.mark.gpu
def test_cv_edge_cases(ctx):
    n, p = 60, 300
    G, y, rng = _panel(29, n, p, 2, effect=0.9)
    ds = _load(ctx, G)
    fold = (np.arange(n) % 2 + 1).astype(np.int32)
    fold[7] = 0                                                # a one-row partition
    res = iht.iht_cv(ds, y, fold, [1, 2])
    assert res.k_best in (1, 2) and np.all(np.isfinite(res.mse)) and res.mse_fold.shape == (3, 2)
    with pytest.raises(iht.IhtError):
        iht.iht_cv(ds, y, np.full(n, 2, np.int32), [1], q=2)       # label out of range
    with pytest.raises(iht.IhtError):
        iht.iht_cv(ds, y, fold, [1], q=4)                           # partition 3 has no rows
    two = np.zeros(n, np.int32)
    two[7] = 1
    with pytest.raises(iht.IhtError):
        iht.iht_cv(ds, y, two, [1])                                 # partition 0 trains on one row
    with pytest.raises(iht.IhtError):
        iht.iht_cv(ds, y, fold, [p + 1])                            # k > p
    bad = y.copy()
    bad[4] = np.nan
    with pytest.raises(iht.IhtError):
        iht.iht_cv(ds, bad, fold, [1, 2])


@pytest.mark.gpu
def test_cv_at_the_simulation_replay_shape(ctx):
    """The Sec. 3.1 replay shape: n = 5289, p = 23 695 (Beta(0.5, 2) allele
    frequencies, 1 % missing), 289 subjects held out (label -1), 5-fold CV on
    the other 5000 over model sizes around the 100-350 of the paper's paths,
    k_true = 200 at SNR 100 %.  Every fold fit the oracle certifies gives the
    oracle's out-of-fold MSE within 1e-4 (11 of the 15 are certified here; the
    other four have a k-th and (k+1)-th |w| closer than the FP32 gradient error
    and are reported as excluded, held only to a sanity bound), the chosen size
    agrees (the curve's minimum is well separated), and the refit is iht_fit on
    the labelled rows."""
    c = synth.CONFIGS[6]
    pn = synth.config_panel(6)
    bed = pn.bed()
    G = oracle.Geno.from_bed(bed, pn.n, pn.p)
    ds = iht.Dataset(ctx, bed, pn.n, pn.p)
    y, causal, beta = synth.phenotype(pn, 200, c["effect_var"], c["noise_var"],
                                      synth.BASE_SEED + 6000 + 17)
    split = np.random.Generator(np.random.PCG64(synth.BASE_SEED + 6000 + 101))
    test = np.sort(split.choice(pn.n, size=c["test"], replace=False)).astype(np.int32)
    train = np.setdiff1d(np.arange(pn.n), test).astype(np.int32)
    fold = np.full(pn.n, -1, np.int32)
    fold[train] = synth.cv_folds(train.size, c["folds"], synth.BASE_SEED + 6007)
    ks = (100, 200, 350)
    res = iht.iht_cv(ds, y, fold, ks, tol=c["tol"], max_iter=c["max_iter"])
    ref = oracle.cv(G, y, fold, c["folds"], ks, tol=c["tol"], max_iter=c["max_iter"], trace=True)
    cert = np.array([[_certified(ref.fits[f][t]) for t in range(len(ks))] for f in range(c["folds"])])
    print(f"[parity] replay-shape CV: {int(cert.sum())} of {cert.size} fold fits certified, "
          f"tie-ambiguous exclusion {1 - cert.mean():.3f}")
    assert int(cert.sum()) == 11
    rel = np.abs(res.mse_fold - ref.mse_fold) / ref.mse_fold
    print(f"[parity] certified fold MSE max rel err {np.max(rel[cert]):.2e}, "
          f"excluded {np.max(rel[~cert]):.2e}")
    assert np.max(rel[cert]) <= BTOL
    assert np.max(rel[~cert]) <= 0.05
    order = np.sort(ref.mse)
    assert order[1] > 1.1 * order[0]                   # a well separated minimum
    assert res.k_best == ref.k_best
    if _certified(ref.fit):
        assert np.array_equal(np.asarray(res.fit.support), ref.fit.support)
        assert res.fit.iterations == ref.fit.iterations
        assert np.max(np.abs(res.fit.beta - ref.fit.beta)) <= BTOL * np.max(np.abs(ref.fit.beta))
    inside = np.flatnonzero(fold >= 0).astype(np.int32)
    alone = iht.iht_fit(ds, y[inside], res.k_best, rows=inside, tol=c["tol"])
    assert np.array_equal(alone.beta, res.fit.beta)
