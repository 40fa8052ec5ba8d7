"""The C-ABI library loads and exports every symbol include/aderdg.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(adg_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_1905_05524_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ["adg_create_mesh", "adg_destroy_mesh", "adg_set_state", "adg_get_state",
                     "adg_predictor", "adg_corrector", "adg_step", "adg_stable_dt",
                     "adg_tv_indicator", "adg_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(built):
    from paper_1905_05524_gb300 import _lib
    assert set(declared_symbols()) <= set(_lib.SIGNATURES), \
        set(declared_symbols()) - set(_lib.SIGNATURES)
    _lib.lib()


def test_last_error_empty_without_calls(built):
    from paper_1905_05524_gb300 import _lib
    assert _lib.lib().adg_last_error() == b""


def test_invalid_descriptor_rejected_without_gpu(built):
    """Argument validation happens before any CUDA call."""
    from paper_1905_05524_gb300 import _lib
    from paper_1905_05524_gb300.solver import MeshConfig
    lib = _lib.lib()
    h = ctypes.c_void_p()
    bad = MeshConfig(degree=9).to_c()
    assert lib.adg_create_mesh(ctypes.byref(bad), ctypes.byref(h)) == _lib.ADG_EINVAL
    assert b"degree" in lib.adg_last_error()
    bad = MeshConfig(nx=0).to_c()
    assert lib.adg_create_mesh(ctypes.byref(bad), ctypes.byref(h)) == _lib.ADG_EINVAL
    assert lib.adg_create_mesh(None, ctypes.byref(h)) == _lib.ADG_EINVAL
    lib.adg_destroy_mesh(None)  # NULL-safe
