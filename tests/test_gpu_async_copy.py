"""State copies with on_device = ADG_COPY_HOST_ASYNC: host memory copied
asynchronously on the caller's stream (no synchronisation inside the call),
for the 2D, finite-volume and 3D meshes; other on_device values are
rejected."""
import ctypes

import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300.solver import FvMesh, Mesh, Mesh3, atmosphere_config, bubble3d_config, fv_bubble_config

pytestmark = pytest.mark.gpu


def roundtrip(setter, getter, h, count, ref):
    s = torch.cuda.Stream()
    sp = ctypes.c_void_p(s.cuda_stream)
    src = ref.cpu().pin_memory()
    dst = torch.empty_like(src).pin_memory()
    L.check(setter(h, ctypes.c_void_p(src.data_ptr()), count, L.ADG_COPY_HOST_ASYNC, sp))
    L.check(getter(h, ctypes.c_void_p(dst.data_ptr()), count, L.ADG_COPY_HOST_ASYNC, sp))
    s.synchronize()
    assert torch.equal(dst, src)
    for bad in (-1, 3):
        with pytest.raises(L.AdgError):
            L.check(setter(h, ctypes.c_void_p(src.data_ptr()), count, bad, sp))
        with pytest.raises(L.AdgError):
            L.check(getter(h, ctypes.c_void_p(dst.data_ptr()), count, bad, sp))


def test_async_host_copies_2d_fv_3d():
    m = Mesh(atmosphere_config(degree=2, nx=5, ny=4))
    u = torch.rand(m.count, dtype=torch.float64) + 1.0
    roundtrip(m._lib.adg_set_state, m._lib.adg_get_state, m.h, m.count, u)
    f = FvMesh(fv_bubble_config(nx=7, ny=6))
    roundtrip(f._lib.adg_fv_set_state, f._lib.adg_fv_get_state, f.h, f.count,
              torch.rand(f.count, dtype=torch.float64))
    g = Mesh3(bubble3d_config(degree=1, n=3))
    roundtrip(g._lib.adg3_set_state, g._lib.adg3_get_state, g.h, g.count,
              torch.rand(g.count, dtype=torch.float64))


def test_async_copy_then_step_matches_synchronous_path():
    cfg = atmosphere_config(degree=3, nx=6, ny=5, precision=L.ADG_PREC_MIXED)
    a, b = Mesh(cfg), Mesh(cfg)
    a.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    u0 = a.get_state().cpu()
    dt = a.stable_dt(0.25)
    a.step(dt, 2)
    s = torch.cuda.Stream()
    sp = ctypes.c_void_p(s.cuda_stream)
    src = u0.pin_memory()
    out = torch.empty_like(src).pin_memory()
    L.check(b._lib.adg_set_state(b.h, ctypes.c_void_p(src.data_ptr()), b.count, L.ADG_COPY_HOST_ASYNC, sp))
    for _ in range(2):
        L.check(b._lib.adg_step(b.h, dt, sp))
    L.check(b._lib.adg_get_state(b.h, ctypes.c_void_p(out.data_ptr()), b.count, L.ADG_COPY_HOST_ASYNC, sp))
    s.synchronize()
    assert torch.equal(out, a.get_state().cpu())
