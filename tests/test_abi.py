"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point that include/gwgb.h declares; host-side argument
validation rejects bad configurations before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "gwgb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gw_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_07660_gb300 import build as b
    b.build()
    from paper_2206_07660_gb300 import load
    return load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "gw_init" in names and "gw_iterate" in names
    for n in names:
        assert hasattr(lib, n), n


def test_init_rejects_bad_config_without_gpu(lib):
    from paper_2206_07660_gb300.gw import GwConfig
    cfg = GwConfig()
    cfg.nao = 0
    out = ctypes.c_void_p()
    dummy = np.zeros(4)
    st = lib.gw_init(ctypes.byref(cfg), dummy.ctypes.data, dummy.ctypes.data, dummy.ctypes.data, ctypes.byref(out))
    assert st == 1 and not out.value
    assert b"positive" in lib.gw_last_error(None)
    st = lib.gw_init(None, None, None, None, ctypes.byref(out))
    assert st == 1
    assert lib.gw_destroy(None) == 1


def test_header_entry_points_documented():
    txt = open(os.path.join(ROOT, "include", "gwgb.h")).read()
    for n in _declared():
        # every entry point is preceded by a comment block
        i = txt.rindex(n + "(")
        assert "*/" in txt[max(0, i - 2000):i], n


def test_library_resolves_every_symbol_at_load():
    """Loading with immediate binding fails on any undefined internal symbol
    (a function declared in a header but defined outside its namespace)."""
    import ctypes
    import os
    from paper_2206_07660_gb300.gw import LIB_PATH
    ctypes.CDLL(LIB_PATH, mode=os.RTLD_NOW)
