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
            names |= set(re.findall(r"\b(adg3?_\w+)\s*\(", txt))
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


def test_header_declares_3d_and_fv_entry_points():
    names = declared_symbols()
    for required in ["adg3_create", "adg3_step", "adg3_stable_dt", "adg3_set_state", "adg3_get_state",
                     "adg_fv_create", "adg_fv_step", "adg_fv_stable_dt"]:
        assert required in names


def test_3d_and_fv_descriptors_rejected_without_gpu(built):
    """The 3D and finite-volume constructors validate their arguments before
    any CUDA call; NULL handles are rejected by every call."""
    from paper_1905_05524_gb300 import _lib
    from paper_1905_05524_gb300.solver import MeshConfig, bubble3d_config, fv_bubble_config
    lib = _lib.lib()
    h = ctypes.c_void_p()
    c3 = bubble3d_config(degree=2, n=3)
    d = c3.to_c()
    # vertical cells, extent, boundary, degree, precision and options
    assert lib.adg3_create(ctypes.byref(d), 0, 0.0, 1000.0, _lib.ADG_BC_WALL, ctypes.byref(h)) == _lib.ADG_EINVAL
    assert lib.adg3_create(ctypes.byref(d), 3, 0.0, -1.0, _lib.ADG_BC_WALL, ctypes.byref(h)) == _lib.ADG_EINVAL
    assert lib.adg3_create(ctypes.byref(d), 3, 0.0, 1000.0, 99, ctypes.byref(h)) == _lib.ADG_EINVAL
    bad = bubble3d_config(degree=_lib.ADG_MAX_DEGREE_3D + 1, n=3).to_c()
    assert lib.adg3_create(ctypes.byref(bad), 3, 0.0, 1000.0, _lib.ADG_BC_WALL, ctypes.byref(h)) == _lib.ADG_EINVAL
    c3.max_levels = 1
    bad = c3.to_c()
    assert lib.adg3_create(ctypes.byref(bad), 3, 0.0, 1000.0, _lib.ADG_BC_WALL,
                           ctypes.byref(h)) == _lib.ADG_EUNSUPPORTED
    c3 = bubble3d_config(degree=2, n=3)
    c3.bc_x, c3.bc_field = _lib.ADG_BC_ANALYTIC, _lib.ADG_FIELD_ABC   # analytic boundaries need gravity off
    bad = c3.to_c()
    assert lib.adg3_create(ctypes.byref(bad), 3, 0.0, 1000.0, _lib.ADG_BC_WALL, ctypes.byref(h)) == _lib.ADG_EINVAL
    assert lib.adg3_create(None, 3, 0.0, 1.0, 0, ctypes.byref(h)) == _lib.ADG_EINVAL
    assert lib.adg3_step(None, 0.1, 1, None) == _lib.ADG_EINVAL
    assert lib.adg3_set_state(None, None, 0, 0, None) == _lib.ADG_EINVAL
    assert lib.adg3_state_count(None) == 0
    lib.adg3_destroy(None)
    # finite volumes: viscosity, boundaries, precision
    cf = fv_bubble_config(nx=8, ny=8)
    cf.mu = 0.01
    bad = cf.to_c()
    assert lib.adg_fv_create(ctypes.byref(bad), ctypes.byref(h)) == _lib.ADG_EINVAL
    cf = fv_bubble_config(nx=8, ny=8)
    cf.precision = 7
    bad = cf.to_c()
    assert lib.adg_fv_create(ctypes.byref(bad), ctypes.byref(h)) == _lib.ADG_EINVAL
    cf = fv_bubble_config(nx=8, ny=8)
    cf.precision, cf.bc_y = _lib.ADG_PREC_MIXED, _lib.ADG_BC_PERIODIC
    bad = cf.to_c()
    assert lib.adg_fv_create(ctypes.byref(bad), ctypes.byref(h)) == _lib.ADG_EUNSUPPORTED
    assert lib.adg_fv_step(None, 0.1, None) == _lib.ADG_EINVAL
    lib.adg_fv_destroy(None)


def test_batch_calls_rejected_without_gpu(built):
    """Batch entry points validate their handle and candidate before touching a device."""
    from paper_1905_05524_gb300 import _lib
    lib = _lib.lib()
    assert lib.adg_batch_set_candidate(None, 0) == _lib.ADG_EINVAL
    assert lib.adg_batch_step(None, None, 1, None) == _lib.ADG_EINVAL
    assert lib.adg_batch_info(None, None, 0) == _lib.ADG_EINVAL
