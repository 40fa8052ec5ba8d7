"""The mixed-precision path at every degree 1-7 against the FP64 oracle.

The packed FP32x2 predictor pairs time slices (for odd n = N+1 the last
pair's second lane repeats a slice against zero-padded weights) and pads
rows to an even length; each degree has its own cells-per-block and
register target.  Stated bound: relative L2 error of theta' <= 1e-6 on the
bubble, and FP32-level error on the periodic manufactured case."""
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300.solver import Mesh, atmosphere_config, steady_manufactured_config
from tests.oracle_bridge import oracle_for, cosine_field, steady_field
from tests.test_gpu_mixed import rel_theta_err, THETA_TOL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("degree", [1, 2, 3, 4, 5, 6, 7])
def test_mixed_bubble_every_degree(degree):
    """Ragged 7x6 walled bubble mesh (the last block of cells is partial),
    12 steps at CFL 0.25."""
    cfg = atmosphere_config(degree=degree, nx=7, ny=6, precision=L.ADG_PREC_MIXED)
    o = oracle_for(cfg)
    u0 = cosine_field(o)
    dt = o.stable_dt(u0, 0.25)
    m = Mesh(cfg)
    m.set_state(u0.cuda().contiguous())
    m.step(dt, 12)
    uo = u0
    for _ in range(12):
        uo = o.step(uo, dt)
    a = m.get_state().cpu()
    err = rel_theta_err(o, a, uo)
    assert err <= THETA_TOL, (degree, err)
    rho = (torch.linalg.vector_norm(a[:, 0] - uo[:, 0]) / torch.linalg.vector_norm(uo[:, 0])).item()
    assert rho <= 1e-9, (degree, rho)


@pytest.mark.parametrize("degree", [1, 2, 4, 6, 7])
def test_mixed_manufactured_every_degree(degree):
    """Periodic steady manufactured field without gravity (the FP32 path
    carries the full state): relative L2 per variable at FP32 level."""
    cfg = steady_manufactured_config(degree=degree, nx=5, ny=4, precision=L.ADG_PREC_MIXED)
    o = oracle_for(cfg)
    u0 = steady_field(o, cfg)
    dt = o.stable_dt(u0, 0.25)
    m = Mesh(cfg)
    m.set_state(u0.cuda().contiguous())
    m.step(dt, 5)
    uo = u0
    for _ in range(5):
        uo = o.step(uo, dt)
    a = m.get_state().cpu()
    for v in range(4):
        r = (torch.linalg.vector_norm(a[:, v] - uo[:, v]) / torch.linalg.vector_norm(uo[:, v])).item()
        assert r <= 1e-6, (degree, v, r)
