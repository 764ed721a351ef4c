"""The allocation-free top-k entry point against the allocating one (needs a GPU).

Some callers cannot allocate device memory (a host that gives all GPU memory to
its own pool, or a loop that must not call cudaMalloc because it can
synchronise the device).  iht_topk_noalloc serves them from a static scratch
array inside the library; this file checks, through the C ABI, that it returns
exactly what iht_topk returns, on two calls in a row (the second call sees the
scratch the first one left behind), and that oversize inputs are refused.
Named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_01398_b300 as iht
    return torch, iht, iht.Context(0)


def test_noalloc_topk_matches_iht_topk_twice(env):
    torch, iht, ctx = env
    rng = np.random.default_rng(20160803)
    cases = [(300_007, 97, "real"), (123_457, 2048, "ties")]
    for p, k, kind in cases:          # two calls in a row on the shared scratch
        if kind == "real":
            w = rng.normal(size=p).astype(np.float32)
        else:
            w = rng.integers(-4, 5, size=p).astype(np.float32)
        wd = torch.from_numpy(w).cuda()
        want = iht.iht_topk(ctx, wd, k).cpu().numpy()
        out = torch.full((k,), -1, dtype=torch.int32, device="cuda")
        iht.iht_topk_noalloc(wd, k, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, want)                 # index work: bit-exact
        ref = np.sort(np.lexsort((np.arange(p), -np.abs(w.astype(np.float64))))[:k])
        assert np.array_equal(got, ref)


def test_noalloc_topk_on_a_side_stream_and_with_nan(env):
    """The call orders its work on the stream it is given; a NaN key ranks above
    +Inf (the call does not synchronise, so it returns no status for it)."""
    torch, iht, ctx = env
    rng = np.random.default_rng(5)
    p, k = 200_003, 64
    w = rng.normal(size=p).astype(np.float32)
    side = torch.cuda.Stream()
    for bad in (None, 1234):
        ww = w.copy()
        if bad is not None:
            ww[bad] = np.nan
        wd = torch.from_numpy(ww).cuda()
        torch.cuda.synchronize()
        out = torch.full((k,), -1, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(side):
            iht.iht_topk_noalloc(wd, k, out, stream=side)
        side.synchronize()
        got = out.cpu().numpy()
        key = np.abs(w.astype(np.float64))
        order = np.lexsort((np.arange(p), -key))
        if bad is not None:                      # the NaN first, then the rest by |w|
            order = np.concatenate([[bad], order[order != bad]])
        assert np.array_equal(got, np.sort(order[:k]))


def test_noalloc_topk_refuses_oversize(env):
    torch, iht, ctx = env
    lib = iht._lib()
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    w = torch.zeros(8, dtype=torch.float32, device="cuda")
    too_big = (1 << 24) + 1              # p beyond the static scratch: refused before any launch
    rc = lib.iht_topk_noalloc(0, None, ctypes.c_void_p(w.data_ptr()), too_big, 4,
                              ctypes.c_void_p(out.data_ptr()))
    assert rc == iht.IHT_EINVAL
    assert lib.iht_topk_noalloc(0, None, ctypes.c_void_p(w.data_ptr()), 8, 9,
                                ctypes.c_void_p(out.data_ptr())) == iht.IHT_EINVAL
