"""Continuous-batching server against the oracle and against itself alone (needs a B300).

Bars: every request the oracle certifies (see test_batch) gets the oracle's
support and iteration count with beta within 1e-4; a request served in a mix
of other requests gives the same support and beta, bit for bit, as when it is
served alone and as iht_fit; admission never holds more device memory than
the budget.
"""
import time

import numpy as np
import pytest

import oracle
from pins import np_Z, random_geno

pytestmark = pytest.mark.gpu

BTOL = 1e-4
GTOL = 1e-5
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


def rel_err(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def certified(fo):
    tr = fo.trace
    return all(tr["gap"][t] > 10 * GTOL * tr["wscale"][t] and not (tr["margin"][t] < 1e-3)
               for t in range(fo.iterations))


def wait_all(srv, tickets, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        if time.time() - t0 > timeout:
            raise TimeoutError(f"{len(tickets) - len(out)} requests still running")
        time.sleep(0.001)
    return [out[t] for t in tickets]


@pytest.fixture(scope="module")
def panel(iht, ctx):
    rng = np.random.default_rng(2024)
    n, p = 900, 4000
    G, codes = random_geno(rng, n, p, miss=0.02)
    ds = iht.Dataset(ctx, np.concatenate([MAGIC, G.body]), n, p)
    Z = np_Z(codes)
    reqs = []
    for r in range(14):
        m = int(rng.integers(450, n + 1))
        rows = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int32)
        ks = int(rng.integers(1, 8))
        causal = rng.choice(p, size=ks, replace=False)
        y = Z[:, causal] @ (rng.choice([-1, 1], size=ks) * 0.6) + rng.normal(size=n)
        k = int(rng.integers(1, 16))
        reqs.append((y[rows] if r % 3 else y, k, rows if r % 3 else None))
    return G, ds, reqs


def test_served_results_match_oracle_and_alone(iht, panel):
    G, ds, reqs = panel
    srv = iht.Server(ds, max_slots=8)
    # a mix: the first half queued at once, the rest arriving while those run
    tickets = [srv.submit(y, k, rows) for (y, k, rows) in reqs[:7]]
    time.sleep(0.002)
    tickets += [srv.submit(y, k, rows) for (y, k, rows) in reqs[7:]]
    mixed = wait_all(srv, tickets)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["active"] == 0 and st["max_active"] <= 8
    assert st["max_active"] >= 2                       # requests did overlap on the device
    # each request alone
    alone = []
    for (y, k, rows) in reqs:
        alone += wait_all(srv, [srv.submit(y, k, rows)])
    srv.close()
    ncert = 0
    for (y, k, rows), a, b in zip(reqs, mixed, alone):
        assert np.array_equal(a.support, b.support)
        assert a.iterations == b.iterations and a.status == b.status
        assert np.array_equal(a.beta_s, b.beta_s)
        fo = oracle.iht(G, y, k, rows=rows)
        if certified(fo):
            ncert += 1
            assert a.iterations == fo.iterations and a.status == fo.status
            assert np.array_equal(a.support, fo.support)
            assert rel_err(a.beta_s, fo.beta[fo.support]) <= BTOL
    print(f"[parity] served requests: {ncert} of {len(reqs)} certified, tie-ambiguous "
          f"exclusion {1 - ncert / len(reqs):.3f}")
    assert ncert == len(reqs)                          # the oracle certifies every request here


def test_served_equals_batched_and_single(iht, panel):
    G, ds, reqs = panel
    srv = iht.Server(ds, max_slots=4)
    served = wait_all(srv, [srv.submit(y, k, rows) for (y, k, rows) in reqs[:5]])
    srv.close()
    batched = iht.iht_fit_batch(ds, reqs[:5])
    for (y, k, rows), a, b in zip(reqs[:5], served, batched):
        assert np.array_equal(a.support, b.support)
        assert np.array_equal(a.beta_s, b.beta_s)
        s = iht.iht_fit(ds, y, k, rows=rows)                # the single-solve path, bit for bit
        assert np.array_equal(a.support, s.support)
        assert np.array_equal(a.beta_s, s.beta[s.support])
        assert a.iterations == s.iterations and a.status == s.status


def test_admission_by_device_footprint(iht, panel):
    G, ds, reqs = panel
    probe = iht.Server(ds, max_slots=4)
    wait_all(probe, [probe.submit(*reqs[0])])
    fp = probe.stats()["max_bytes_in_use"]
    probe.close()
    assert fp > 0
    # room for two solves of this size: the rest wait for memory, not for slots
    y, k, rows = reqs[0]
    srv = iht.Server(ds, max_slots=16, hbm_budget=int(2.5 * fp))
    res = wait_all(srv, [srv.submit(y, k, rows) for _ in range(6)])
    st = srv.stats()
    srv.close()
    assert st["completed"] == 6 and st["max_active"] <= 2
    assert st["max_bytes_in_use"] <= int(2.5 * fp)
    for r in res[1:]:
        assert np.array_equal(r.support, res[0].support)
        assert np.array_equal(r.beta_s, res[0].beta_s)


def test_server_errors(iht, panel):
    G, ds, reqs = panel
    srv = iht.Server(ds, max_slots=4, hbm_budget=0)
    y, k, rows = reqs[1]
    bad = y.copy()
    bad[5] = np.nan
    t_nan = srv.submit(bad, 4, rows)
    dup = np.array([3, 3, 7, 9], np.int32)
    t_dup = srv.submit(np.ones(4), 2, dup)
    t_ok = srv.submit(y, k, rows)
    r_nan, r_dup, r_ok = wait_all(srv, [t_nan, t_dup, t_ok])
    assert r_nan.status == iht.IHT_ENUMERIC and r_nan.iterations == 0
    assert r_dup.status == iht.IHT_EINVAL
    assert r_ok.status in (iht.IHT_OK, iht.IHT_ENOTCONV) and r_ok.iterations > 0
    with pytest.raises(iht.IhtError):
        srv.submit(y, ds.p + 1, rows)                       # k > p
    with pytest.raises(iht.IhtError):
        srv.submit(y[:1], 1, rows[:1])                      # n_rows < 2
    srv._k[999999] = 1
    with pytest.raises(iht.IhtError):
        srv.poll(999999)                                    # unknown ticket
    srv.close()
    tiny = iht.Server(ds, max_slots=2, hbm_budget=4096)
    with pytest.raises(iht.IhtError):
        tiny.submit(y, k, rows)                             # can never fit the budget
    tiny.close()
