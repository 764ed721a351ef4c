"""The shared input generator: layout, determinism and the drawn distributions."""
import numpy as np

import oracle
import synth
from pins import py_decode


def test_bed_layout_matches_codes():
    pn = synth.panel(37, 11, seed=3, miss=0.05)
    bed = pn.bed()
    assert bytes(bed[:3]) == synth.BED_MAGIC
    rb = pn.bed_row_bytes
    dec = py_decode(bed[3:], pn.n, pn.p, rb)
    assert np.array_equal(dec, pn.codes(np.arange(pn.p)))
    # pad bits of the last byte are zero
    last = bed[3:].reshape(pn.p, rb)[:, -1]
    assert np.all((last >> 2) == 0)        # n = 37 -> one sample in the last byte


def test_padded_rows_and_ranges():
    pn = synth.panel(10, 9, seed=4)
    full = pn.bed_body(row_bytes=16).reshape(9, 16)
    assert np.all(full[:, 3:] == 0)
    part = pn.bed_body(3, 7).reshape(4, 3)
    assert np.array_equal(part, pn.bed_body().reshape(9, 3)[3:7])


def test_deterministic_and_distribution():
    a = synth.panel(4000, 50, seed=9, miss=0.01)
    b = synth.panel(4000, 50, seed=9, miss=0.01)
    assert np.array_equal(a.bed(), b.bed())
    c = a.codes(np.arange(50))
    miss = np.mean(c == 1)
    assert 0.007 < miss < 0.013
    obs = c != 1
    dose = np.select([c == 2, c == 3], [1.0, 2.0], 0.0)
    freq = (dose * obs).sum(1) / (2 * obs.sum(1))
    assert np.max(np.abs(freq - a.maf)) < 0.03


def test_phenotype_uses_population_frequency():
    pn = synth.panel(3000, 200, seed=5)
    y, causal, beta = synth.phenotype(pn, 5, 0.25, 1.0, seed=6)
    assert y.shape == (3000,) and causal.size == 5 and np.all(np.diff(causal) > 0)
    y2, causal2, _ = synth.phenotype(pn, 5, 0.25, 1.0, seed=6)
    assert np.array_equal(y, y2) and np.array_equal(causal, causal2)
    # h2 rescaling hits its target on the realised signal
    y3, c3, b3 = synth.phenotype(pn, 20, 1.0, 1.0, seed=7, h2=0.4)
    z = synth._pop_standardised(pn, c3, None)
    s = z @ b3
    assert abs(np.var(s) / (np.var(s) + 1.0) - 0.4) < 1e-9
