"""The FP64 oracle against its pins (CPU only)."""
import numpy as np
import pytest

import oracle
import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.load())


def test_status_codes():
    G = pins.geno_from_codes(np.array([[0, 2, 3, 0], [3, 2, 0, 2]], dtype=np.int8))
    y = np.array([1.0, 2.0, np.nan, 0.0])
    assert oracle.iht(G, y, 1).status == oracle.ENUMERIC
    with pytest.raises(RuntimeError):
        oracle.iht(G, np.zeros(4), 3)          # k > p
    f = oracle.iht(G, np.zeros(4), 1)           # g = 0 everywhere: converged at once
    assert f.status == oracle.OK and f.iterations == 0 and not f.beta.any()


def test_thread_count_does_not_change_results():
    rng = np.random.default_rng(5)
    G, codes = pins.random_geno(rng, 90, 200, miss=0.02)
    y = rng.normal(size=G.n)
    oracle.set_threads(1)
    a = oracle.iht(G, y, 7)
    oracle.set_threads(4)
    b = oracle.iht(G, y, 7)
    assert np.array_equal(a.beta, b.beta) and a.iterations == b.iterations
