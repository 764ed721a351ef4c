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
    assert o.variant == iht.IHT_VARIANT_IHT
    assert o.flags == 0
    assert ctypes.sizeof(iht.iht_options) == 56 and ctypes.sizeof(iht.iht_result) == 48
    assert lib.iht_kernel_launches() == 0


def test_argument_checks_need_no_device():
    lib = iht._lib()
    assert lib.iht_create(None, 0, None) == iht.IHT_EINVAL
    assert lib.iht_destroy(None) == iht.IHT_EINVAL
    assert lib.iht_dataset_free(None) == iht.IHT_EINVAL
    assert lib.iht_fit(None, None, 0, None, 1, None, None, None, None) == iht.IHT_EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of the public structs have the C layout (sizes and offsets)."""
    import subprocess
    structs = {"iht_options": iht.iht_options, "iht_result": iht.iht_result,
               "iht_trace": iht.iht_trace, "iht_solve_desc": iht.iht_solve_desc,
               "iht_server_options": iht.iht_server_options,
               "iht_server_stats": iht.iht_server_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "iht.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    got = {(a, b): int(c) for a, b, c in (l.split() for l in out if l)}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def test_server_entry_points_check_arguments():
    lib = iht._lib()
    o = iht.iht_server_options()
    lib.iht_server_default_options(ctypes.byref(o))
    assert o.max_slots == 64 and o.hbm_budget == 0 and o.solve.max_iter == 100
    assert lib.iht_server_create(None, ctypes.byref(o), None) == iht.IHT_EINVAL
    assert lib.iht_server_submit(None, None, None) == iht.IHT_EINVAL
    assert lib.iht_server_poll(None, 1, None, None, None, None) == iht.IHT_EINVAL
    assert lib.iht_server_get_stats(None, None) == iht.IHT_EINVAL
    assert lib.iht_server_destroy(None) == iht.IHT_EINVAL


def test_fault_injection_arguments():
    """Host-side fault injection checks its arguments and needs no device."""
    lib = iht._lib()
    assert lib.iht_fault_inject(iht.IHT_FAULT_NONE, 0) == iht.IHT_OK
    assert lib.iht_fault_inject(3, 1) == iht.IHT_EINVAL
    assert lib.iht_fault_inject(iht.IHT_FAULT_ALLOC, -1) == iht.IHT_EINVAL
    assert lib.iht_fault_inject(iht.IHT_FAULT_TIMEOUT, 2) == iht.IHT_OK
    assert lib.iht_fault_inject(iht.IHT_FAULT_NONE, 0) == iht.IHT_OK
