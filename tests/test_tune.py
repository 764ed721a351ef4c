"""Launch shapes of the gradient passes and their autotuner.

A shape changes only how genotype and residual tiles are staged (TMA stages of
the single-column pass; genotype stages, buffer pairs and the finalisation
width of the multi-column pass), never the arithmetic of Sec. 2.2's
g = Z^T r or its order, so every shape must give the same bits, and the tuned
choice the same bits as any pinned one.  Argument checks run on the host.
"""
import itertools

import numpy as np
import pytest

import paper_1608_01398_b300 as iht
from pins import random_geno

MAGIC = np.array([0x6C, 0x1B, 0x01], dtype=np.uint8)


def test_tuning_api_on_the_host():
    L = iht._lib()
    iht.tune_clear()
    assert iht.tuning_summary() == ""
    assert L.iht_tuning_summary(None, 0) == 1
    iht.set_autotune(False)
    iht.set_autotune(True)
    prm = np.array([4, 1, 1, 1, 2], np.int32)
    assert L.iht_tune_pin(None, iht.IHT_PASS_MULTI, 8, prm.ctypes.data, 5) == iht.IHT_EINVAL
    assert L.iht_tune_query(None, iht.IHT_PASS_MULTI, 8, prm.ctypes.data, 5) == iht.IHT_EINVAL


# --------------------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def panel():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = iht.Context(0)
    rng = np.random.default_rng(23)
    n, p = 1500, 3000                         # 12 tiles of 256 SNPs and a ragged one
    G, _ = random_geno(rng, n, p, miss=0.02)
    ds = iht.Dataset(ctx, np.concatenate([MAGIC, G.body]), n, p)
    R = [torch.from_numpy(rng.normal(size=n).astype(np.float32)).cuda() for _ in range(44)]
    yield ds, R
    iht.tune_clear()
    iht.set_autotune(True)


def _single(ds, r):
    return iht.iht_gradient(ds, r, impl=2).cpu().numpy()


@pytest.mark.gpu
def test_single_column_stage_counts_give_the_same_bits(panel):
    ds, R = panel
    iht.tune_clear()
    outs = []
    for nst in range(2, 9):
        try:
            iht.tune_pin(ds, iht.IHT_PASS_SINGLE, 1, [nst])
        except iht.IhtError:                   # more stages than shared memory holds
            assert nst > 2
            break
        assert iht.tune_query(ds, iht.IHT_PASS_SINGLE, 1) == (nst,)
        outs.append(_single(ds, R[0]))
    assert len(outs) >= 2
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    with pytest.raises(iht.IhtError):
        iht.tune_pin(ds, iht.IHT_PASS_SINGLE, 1, [1])
    iht.tune_clear()


@pytest.mark.gpu
@pytest.mark.parametrize("ncols", [6, 20, 30, 44])
def test_multi_column_shapes_give_the_same_bits(panel, ncols):
    ds, R = panel
    iht.tune_clear()
    want = np.stack([_single(ds, R[c]) for c in range(ncols)])
    tried = 0
    for tiles, ngs, pairs, fin8, padded in itertools.product((2, 4), (2, 4, 6, 8), (0, 1), (0, 1), (0, 1)):
        try:
            iht.tune_pin(ds, iht.IHT_PASS_MULTI, ncols, [ngs, pairs, fin8, padded, tiles])
        except iht.IhtError:
            # pairs need four or more A buffers; 4 tiles need N <= 96 and at most
            # 6 genotype stages beside the B chunks
            assert (pairs == 1 and ncols > 38) or (tiles == 4 and (ncols > 19 or ngs > 6 or
                                                                   (pairs == 1 and ncols > 12)))
            continue
        got = iht.iht_gradient_batch(ds, R[:ncols], impl=2).cpu().numpy()
        assert np.array_equal(got, want), (tiles, ngs, pairs, fin8, padded)
        tried += 1
    assert tried >= 16
    with pytest.raises(iht.IhtError):
        iht.tune_pin(ds, iht.IHT_PASS_MULTI, ncols, [9, 0, 0, 0, 2])
    with pytest.raises(iht.IhtError):
        iht.tune_pin(ds, iht.IHT_PASS_MULTI, ncols, [4, 0, 0, 2, 2])
    with pytest.raises(iht.IhtError):
        iht.tune_pin(ds, iht.IHT_PASS_MULTI, ncols, [4, 0, 0, 0, 3])
    iht.tune_clear()


@pytest.mark.gpu
def test_tuner_caches_a_shape_and_keeps_the_bits(panel):
    ds, R = panel
    iht.tune_clear()
    iht.set_autotune(False)
    want1 = _single(ds, R[3])
    want = iht.iht_gradient_batch(ds, R[:20], impl=2).cpu().numpy()
    assert iht.tune_query(ds, iht.IHT_PASS_MULTI, 20) is None       # off: default shape, nothing cached
    assert iht.tune_query(ds, iht.IHT_PASS_SINGLE, 1) is None
    iht.set_autotune(True)
    got1 = _single(ds, R[3])                                         # tunes, then cached
    got = iht.iht_gradient_batch(ds, R[:20], impl=2).cpu().numpy()
    assert np.array_equal(got1, want1) and np.array_equal(got, want)
    nst, = iht.tune_query(ds, iht.IHT_PASS_SINGLE, 1)
    ngs, pairs, fin8, padded, tiles = iht.tune_query(ds, iht.IHT_PASS_MULTI, 20)
    assert nst >= 2 and ngs in (4, 6, 8) and pairs in (0, 1) and fin8 in (0, 1) and padded in (0, 1)
    assert tiles in (2, 4)
    assert iht.tune_query(ds, iht.IHT_PASS_MULTI, 21) == (ngs, pairs, fin8, padded, tiles)  # same bucket
    assert iht.tune_query(ds, iht.IHT_PASS_MULTI, 40) is None                  # another bucket
    text = iht.tuning_summary()
    assert "single-column" in text and "multi-column" in text and "tuned" in text
    again = iht.iht_gradient_batch(ds, R[:20], impl=2).cpu().numpy()          # cached shape
    assert np.array_equal(again, want)
    iht.tune_clear()
