"""The C ABI library builds, loads and exports every function that include/*.h declares (CPU only)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(bz_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    return __graft_entry__._libbuild().build()


def test_header_declares_functions():
    assert "bz_collide" in _declared() and "bz_plan_create" in _declared()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_argument_checks_without_gpu(libpath):
    import paper_2004_11239_gb300 as bz
    assert bz.bz_status_str(0) == "ok"
    assert bz.bz_status_str(1) == "invalid argument"
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    assert bz.lib.bz_plan_create(ctypes.byref(h), 20, 10.0, 9.0, 0.0, 0.5, 4, 12) == 1   # N = 20
    assert bz.lib.bz_plan_create(ctypes.byref(h), 16, -1.0, 9.0, 0.0, 0.5, 4, 12) == 1   # L < 0
    assert bz.lib.bz_collide(None, None, None, 0, None) == 1
    assert h.value is None
