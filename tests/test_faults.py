"""How failures reach the caller, with the failure made on the host (needs a B300).

No device fault, trap or hang is made.  iht_fault_inject makes the library's
next device allocation fail as on an exhausted device, or writes a gradient
pass's bounded-wait error word from the host before the library reads it (as a
device wait that gave up would leave it).  Every entry point that allocates or
runs a tensor-core pass must then return ENOMEM or ETIMEOUT, release what it
took, and work normally on the next call.
"""
import time

import numpy as np
import pytest

from pins import random_geno

pytestmark = pytest.mark.gpu

MAGIC = np.array([0x6C, 0x1B, 0x01], dtype=np.uint8)


@pytest.fixture(scope="module")
def iht():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_01398_b300 as m
    yield m
    m.fault_inject(m.IHT_FAULT_NONE)


@pytest.fixture(scope="module")
def ctx(iht):
    return iht.Context(0)


@pytest.fixture(scope="module")
def panel():
    rng = np.random.default_rng(77)
    G, _ = random_geno(rng, 600, 900, miss=0.02)
    y = rng.normal(size=600)
    return G, y


def fresh(iht, ctx, G):
    return iht.Dataset(ctx, np.concatenate([MAGIC, G.body]), G.n, G.p)


def status_of(fn):
    try:
        fn()
    except Exception as e:          # IhtError carries the status
        return getattr(e, "status", None)
    return 0


def test_alloc_failure_in_fit_then_recovery(iht, ctx, panel):
    G, y = panel
    ds = fresh(iht, ctx, G)           # no workspace yet: the first fit allocates it
    iht.fault_inject(iht.IHT_FAULT_ALLOC, 1)
    assert status_of(lambda: iht.iht_fit(ds, y, 7)) == iht.IHT_ENOMEM
    iht.fault_inject(iht.IHT_FAULT_NONE)
    a = iht.iht_fit(ds, y, 7)
    b = iht.iht_fit(fresh(iht, ctx, G), y, 7)
    assert a.status in (iht.IHT_OK, iht.IHT_ENOTCONV)
    assert np.array_equal(a.beta, b.beta) and a.iterations == b.iterations


def test_alloc_failure_in_batch_then_recovery(iht, ctx, panel):
    G, y = panel
    ds = fresh(iht, ctx, G)
    iht.iht_fit(ds, y, 5)                              # workspace in place; batch work is not
    probs = [(y, 5, None), (y[::-1].copy(), 9, None)]
    iht.fault_inject(iht.IHT_FAULT_ALLOC, 1)
    assert status_of(lambda: iht.iht_fit_batch(ds, probs)) == iht.IHT_ENOMEM
    iht.fault_inject(iht.IHT_FAULT_NONE)
    out = iht.iht_fit_batch(ds, probs)
    alone = iht.iht_fit(ds, y, 5)
    assert np.array_equal(out[0].beta, alone.beta)


def test_alloc_failure_in_server_admission(iht, ctx, panel):
    G, y = panel
    ds = fresh(iht, ctx, G)
    srv = iht.Server(ds, max_slots=4)
    iht.fault_inject(iht.IHT_FAULT_ALLOC, 1)           # the admitted request's device block
    t = srv.submit(y, 6)
    t0, st = time.time(), None
    while st is None and time.time() - t0 < 60:
        try:
            if srv.poll(t) is not None:
                st = 0
        except iht.IhtError as e:
            st = e.status
        time.sleep(0.002)
    iht.fault_inject(iht.IHT_FAULT_NONE)
    assert st == iht.IHT_ENOMEM
    srv.close()
    srv2 = iht.Server(ds, max_slots=4)                 # a new server works
    t2 = srv2.submit(y, 6)
    r = None
    t0 = time.time()
    while r is None and time.time() - t0 < 60:
        r = srv2.poll(t2)
        time.sleep(0.002)
    srv2.close()
    assert r is not None and r.status in (iht.IHT_OK, iht.IHT_ENOTCONV)


def test_timeout_word_reaches_every_entry_point(iht, ctx, panel):
    import torch
    G, y = panel
    ds = fresh(iht, ctx, G)
    ref = iht.iht_fit(ds, y, 7)
    r = torch.from_numpy(np.random.default_rng(1).normal(size=G.n).astype(np.float32)).cuda()
    calls = {
        "iht_fit": lambda: iht.iht_fit(ds, y, 7),
        "iht_fit_trace": lambda: iht.iht_fit_trace(ds, y, 7),
        "iht_gradient": lambda: iht.iht_gradient(ds, r),
        "iht_fit_batch": lambda: iht.iht_fit_batch(ds, [(y, 7, None), (y, 4, None)]),
        "iht_gradient_batch": lambda: iht.iht_gradient_batch(ds, [r, r, r], impl=2),
        "iht_cv": lambda: iht.iht_cv(ds, y, np.arange(G.n) % 3, [2, 4]),
    }
    for name, fn in calls.items():
        fn()                                            # the pass has run once: its word exists
        iht.fault_inject(iht.IHT_FAULT_TIMEOUT, 1)
        got = status_of(fn)
        iht.fault_inject(iht.IHT_FAULT_NONE)
        assert got == iht.IHT_ETIMEOUT, name
        assert status_of(fn) == 0, f"{name} after the injected timeout"
    again = iht.iht_fit(ds, y, 7)
    assert np.array_equal(again.beta, ref.beta)


def test_timeout_word_stops_the_server(iht, ctx, panel):
    G, y = panel
    ds = fresh(iht, ctx, G)
    srv = iht.Server(ds, max_slots=4, tol=1e-12, max_iter=40)   # >= 16 ticks: one status read
    iht.fault_inject(iht.IHT_FAULT_TIMEOUT, 1)
    t = srv.submit(y, 6)
    t0, st = time.time(), None
    while st is None and time.time() - t0 < 60:
        try:
            if srv.poll(t) is not None:
                st = 0
        except iht.IhtError as e:
            st = e.status
        time.sleep(0.002)
    iht.fault_inject(iht.IHT_FAULT_NONE)
    srv.close()
    assert st == iht.IHT_ETIMEOUT
