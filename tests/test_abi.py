"""The C-ABI library builds, loads and exports every entry point of include/iht.h (CPU only)."""
import ctypes
import os
import re

import paper_1608_01398_b300 as iht

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "iht.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(iht_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = iht._lib()
    names = declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(iht.EXPORTED)


def test_host_only_entry_points():
    lib = iht._lib()
    for s in range(8):
        assert lib.iht_strerror(s)
    o = iht.iht_default_options()
    assert (o.max_iter, o.max_backtrack, o.tol, o.c, o.kappa) == (100, 50, 1e-4, 0.01, 2.0)
    assert ctypes.sizeof(iht.iht_options) == 48 and ctypes.sizeof(iht.iht_result) == 48
    assert lib.iht_kernel_launches() == 0


def test_argument_checks_need_no_device():
    lib = iht._lib()
    assert lib.iht_create(None, 0, None) == iht.IHT_EINVAL
    assert lib.iht_destroy(None) == iht.IHT_EINVAL
    assert lib.iht_dataset_free(None) == iht.IHT_EINVAL
    assert lib.iht_fit(None, None, 0, None, 1, None, None, None, None) == iht.IHT_EINVAL
