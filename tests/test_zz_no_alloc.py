"""adg_step_noalloc: the allocation-free step entry point.

Some callers cannot call cudaMalloc (their pool allocator owns the device
memory, or a latency-critical loop cannot take cudaMalloc's device-wide
synchronisation).  For them adg_step_noalloc runs the same FP64 step as
adg_step on a caller-owned state, with its scratch in a fixed static device
array instead of a mesh workspace.  This test calls it through the C ABI
twice in a row and checks each result against the existing entry point
(adg_step through a mesh) within the FP64 parity tolerance of the other
tests.  It lives in its own file, collected last, and works both alone in a
fresh process and after the other tests."""
import ctypes

import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300.solver import Mesh, atmosphere_config, steady_manufactured_config
from tests.tolerances import momentum_floor

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _close(a, b, floor):
    """Per-variable L2 within TOL of the reference, plus the momentum
    rounding floor of tests/tolerances.py for a fluid near rest over a
    hydrostatic background."""
    for v in range(4):
        d = torch.linalg.vector_norm(a[:, v] - b[:, v]).item()
        nb = torch.linalg.vector_norm(b[:, v]).item()
        bound = TOL * nb + (floor if v in (1, 2) else 0.0)
        assert d <= bound, (v, d, bound)


@pytest.mark.parametrize("cfg", [steady_manufactured_config(degree=3, nx=9, ny=9),
                                 atmosphere_config(degree=5, nx=27, ny=27)])
def test_noalloc_step_matches_mesh_step_twice(cfg):
    lib = L.lib()
    ref = Mesh(cfg)
    if cfg.gravity:
        ref.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
        dt = ref.stable_dt(0.25)
    else:
        ref.init_scenario(L.ADG_SCEN_STEADY)
        dt = ref.stable_dt(0.5)
    u = ref.get_state().clone()            # caller-owned state for the no-alloc path
    desc = cfg.to_c()
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    for k in range(2):                     # two calls in a row
        ref.step(dt)
        L.check(lib.adg_step_noalloc(ctypes.byref(desc), ctypes.c_void_p(u.data_ptr()), u.numel(),
                                     float(dt), sp))
        torch.cuda.synchronize()
        _close(u.cpu(), ref.get_state().cpu(), momentum_floor(cfg, dt, k + 1, u[:, 0].numel()))
    ref.close()


def test_noalloc_rejects_oversized_mesh_and_bad_count():
    lib = L.lib()
    big = atmosphere_config(degree=5, nx=200, ny=200)
    desc = big.to_c()
    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = 200 * 200 * 36 * 4
    rc = lib.adg_step_noalloc(ctypes.byref(desc), ctypes.c_void_p(u.data_ptr()), n, 0.01, sp)
    assert rc == L.ADG_EINVAL
    assert b"static limit" in lib.adg_last_error()
    small = steady_manufactured_config(degree=2, nx=3, ny=3).to_c()
    rc = lib.adg_step_noalloc(ctypes.byref(small), ctypes.c_void_p(u.data_ptr()), 5, 0.01, sp)
    assert rc == L.ADG_EINVAL
    # an adaptive-mesh description is refused rather than stepped as a uniform mesh
    amr = steady_manufactured_config(degree=2, nx=3, ny=3)
    amr.max_levels = 1
    rc = lib.adg_step_noalloc(ctypes.byref(amr.to_c()), ctypes.c_void_p(u.data_ptr()), 3 * 3 * 9 * 4, 0.01, sp)
    assert rc == L.ADG_EUNSUPPORTED
    # absurd sizes are refused before any size arithmetic can wrap
    huge = steady_manufactured_config(degree=2, nx=1 << 20, ny=1 << 20).to_c()
    rc = lib.adg_step_noalloc(ctypes.byref(huge), ctypes.c_void_p(u.data_ptr()), 36, 0.01, sp)
    assert rc == L.ADG_EINVAL and b"2^26" in lib.adg_last_error()
    assert torch.cuda.current_device() == 0
