"""The C-ABI library builds, loads and exports every symbol of include/fblts.h (no GPU needed)."""
import os
import re

import pytest

import paper_2405_10505_gb300 as fb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fblts.h")).read()
    return sorted(set(re.findall(r"^(?:fblts_status|const char \*)\s*(fblts_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported():
    L = fb.lib()
    names = _declared()
    assert "fblts_lts_advance" in names and "fblts_mesh_create" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(fb.SYMBOLS)


def test_errors_are_reported_not_raised_in_c():
    L = fb.lib()
    import ctypes as C
    h = C.c_void_p()
    assert L.fblts_mesh_create(None, C.byref(h)) == fb.E_ARG
    assert "NULL" in fb.last_error()


def test_bad_sizes_rejected_before_device_use():
    d = fb.MeshDesc()
    import ctypes as C
    h = C.c_void_p()
    assert fb.lib().fblts_mesh_create(C.byref(d), C.byref(h)) == fb.E_ARG
