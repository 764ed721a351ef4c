"""Checkpoint / resume: the solve-state image and resumed solves.

Between iterations IHT carries only S, beta on S and its counters (Sec. 2.2:
r, g and the step size are recomputed from them), so a solve stopped after m
iterations and resumed from its image must take exactly the iterations of the
uninterrupted solve.  The image tests run on the host through the C ABI (no
GPU); the resume tests need a B300.
"""
import ctypes

import numpy as np
import pytest

import paper_1608_01398_b300 as iht
from pins import np_Z, random_geno

MAGIC = np.array([0x6C, 0x1B, 0x01], dtype=np.uint8)


def _fake_fit(rng, p, k):
    supp = np.sort(rng.choice(p, size=k, replace=False)).astype(np.int32)
    beta = np.zeros(p)
    beta[supp] = rng.normal(size=k)
    return iht.FitResult(beta, supp, 7, iht.IHT_ENOTCONV, 3, 12.5, 0.25)


def test_state_round_trip_on_host():
    rng = np.random.default_rng(1)
    for k in (1, 5, 200):
        fit = _fake_fit(rng, 5000, k)
        img = iht.save_state((900, 5000), 850, fit)
        size = ctypes.c_size_t()
        assert iht._lib().iht_state_bytes(k, ctypes.byref(size)) == iht.IHT_OK
        assert len(img) == size.value == 80 + 12 * k
        st = iht.load_state(img)
        assert (st.n, st.p, st.n_rows, st.k) == (900, 5000, 850, k)
        assert np.array_equal(st.support, fit.support)
        assert np.array_equal(st.beta_s, fit.beta[fit.support])
        assert (st.iterations, st.backtracks, st.status) == (7, 3, iht.IHT_ENOTCONV)
        assert (st.objective, st.mu) == (12.5, 0.25)


def test_state_rejects_damaged_images():
    rng = np.random.default_rng(2)
    img = bytearray(iht.save_state((900, 5000), 900, _fake_fit(rng, 5000, 9)))
    for pos in (0, 8, 20, 48, 60, 80, 100, len(img) - 1):     # magic, version, shape, counters, arrays
        bad = bytearray(img)
        bad[pos] ^= 0x40
        with pytest.raises(iht.IhtError):
            iht.load_state(bytes(bad))
    with pytest.raises(iht.IhtError):
        iht.load_state(bytes(img[:-1]))                       # truncated
    with pytest.raises(iht.IhtError):
        iht.load_state(bytes(img) + b"\0")                    # trailing bytes
    with pytest.raises(iht.IhtError):
        iht.load_state(b"")


def test_state_save_rejects_invalid_contents():
    rng = np.random.default_rng(3)
    fit = _fake_fit(rng, 100, 4)
    unsorted = iht.FitResult(fit.beta, fit.support[::-1].copy(), 1, 0, 0, 0.0, 0.0)
    with pytest.raises(iht.IhtError):
        iht.save_state((50, 100), 50, unsorted)
    nan = iht.FitResult(fit.beta.copy(), fit.support, 1, 0, 0, 0.0, 0.0)
    nan.beta[fit.support[0]] = np.nan
    with pytest.raises(iht.IhtError):
        iht.save_state((50, 100), 50, nan)
    with pytest.raises(iht.IhtError):
        iht.save_state((50, 100), 51, fit)                    # more rows than the dataset
    out_of_range = iht.FitResult(fit.beta, np.array([1, 2, 3, 100], np.int32), 1, 0, 0, 0.0, 0.0)
    out_of_range.beta_s = np.ones(4)
    with pytest.raises(iht.IhtError):
        iht.save_state((50, 100), 50, out_of_range)


# --------------------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def gpu_panel():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = iht.Context(0)
    rng = np.random.default_rng(7)
    n, p = 1200, 6000
    G, codes = random_geno(rng, n, p, miss=0.02)
    ds = iht.Dataset(ctx, np.concatenate([MAGIC, G.body]), n, p)
    Z = np_Z(codes)                                            # n x p, standardised
    causal = rng.choice(p, size=12, replace=False)
    y = Z[:, causal] @ rng.normal(size=12) * 0.3 + rng.normal(size=n)
    return ctx, ds, y, rng


@pytest.mark.gpu
@pytest.mark.parametrize("m", [1, 2, 5])
def test_resumed_solve_equals_uninterrupted(gpu_panel, m):
    ctx, ds, y, rng = gpu_panel
    k = 20
    full = iht.iht_fit(ds, y, k, max_iter=100)
    assert full.iterations > m
    part = iht.iht_fit(ds, y, k, max_iter=m)
    assert part.status == iht.IHT_ENOTCONV and part.iterations == m
    img = iht.save_state(ds, ds.n, part)
    res = iht.iht_fit_resume(ds, y, img, max_iter=100)
    assert np.array_equal(res.support, full.support)
    assert np.array_equal(res.beta, full.beta)                 # bit for bit
    assert (res.iterations, res.status, res.backtracks) == (full.iterations, full.status,
                                                            full.backtracks)
    assert res.objective == full.objective


@pytest.mark.gpu
def test_resume_on_a_row_subset_and_chained(gpu_panel):
    ctx, ds, y, rng = gpu_panel
    rows = np.sort(rng.choice(ds.n, size=1000, replace=False)).astype(np.int32)
    yr, k = y[rows], 15
    full = iht.iht_fit(ds, yr, k, rows=rows, max_iter=100)
    img, total = None, 0
    while True:                                                # one iteration per call
        total += 1
        f = (iht.iht_fit(ds, yr, k, rows=rows, max_iter=1) if img is None
             else iht.iht_fit_resume(ds, yr, img, rows=rows, max_iter=total))
        img = iht.save_state(ds, rows.size, f)
        if f.status != iht.IHT_ENOTCONV or total >= 100:
            break
    assert np.array_equal(f.support, full.support) and np.array_equal(f.beta, full.beta)
    assert f.iterations == full.iterations and f.status == full.status


@pytest.mark.gpu
def test_resume_checks_the_image_against_the_solve(gpu_panel):
    ctx, ds, y, rng = gpu_panel
    part = iht.iht_fit(ds, y, 10, max_iter=2)
    img = iht.save_state(ds, ds.n, part)
    rows = np.arange(ds.n - 1, dtype=np.int32)
    with pytest.raises(iht.IhtError):                          # fitted on n rows, resumed on n-1
        iht.iht_fit_resume(ds, y[:-1], img, rows=rows)
    other = iht.save_state((ds.n, ds.p + 1), ds.n, part)
    with pytest.raises(iht.IhtError):                          # another dataset's shape
        iht.iht_fit_resume(ds, y, other)
    same = iht.iht_fit_resume(ds, y, img, max_iter=2)          # nothing left to do
    assert same.iterations == 2 and np.array_equal(same.beta, part.beta)
