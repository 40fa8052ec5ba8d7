"""Parity at the degree-sweep size (243 x 243 periodic cells, steady
manufactured problem, degrees 2-7, FP64 and mixed) on sampled windows.

One step of a cell depends only on its own state and its four neighbours
(the predictor is element-local, the corrector reads the neighbours'
traces), so the oracle stepping a 7 x 7 window of the full state (with the
window's own coordinates) reproduces the full mesh's step on the window's
inner 5 x 5 cells exactly: compared there at 1e-11 (FP64) and 1e-6 (mixed,
FP32 level) relative per variable."""
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300.solver import Mesh, steady_manufactured_config
from tests.oracle_bridge import oracle_for

pytestmark = pytest.mark.gpu

NX = 243
WINDOWS = [(0, 0), (117, 58), (236, 236)]


def window(u, wx, wy, w, n):
    U = u.reshape(NX, NX, 4, n, n)
    return U[wy:wy + w, wx:wx + w].reshape(w * w, 4, n, n).contiguous()


@pytest.mark.parametrize("degree", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("prec", [L.ADG_PREC_FP64, L.ADG_PREC_MIXED])
def test_sweep_size_step_on_sampled_windows(degree, prec):
    cfg = steady_manufactured_config(degree=degree, nx=NX, ny=NX, precision=prec)
    n = degree + 1
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_STEADY)
    u0 = m.get_state().cpu()
    dt = m.stable_dt(0.5)
    m.step(dt)
    u1 = m.get_state().cpu()
    h = cfg.Lx / NX
    tol = 1e-11 if prec == L.ADG_PREC_FP64 else 1e-6
    for wx, wy in WINDOWS:
        wc = steady_manufactured_config(degree=degree, nx=7, ny=7)
        wc.x0, wc.y0, wc.Lx, wc.Ly = wx * h, wy * h, 7 * h, 7 * h
        o = oracle_for(wc)
        uo = o.step(window(u0, wx, wy, 7, n), dt, 0.0)
        a = window(u1, wx, wy, 7, n).reshape(7, 7, 4, n, n)[1:6, 1:6]
        b = uo.reshape(7, 7, 4, n, n)[1:6, 1:6]
        for v in range(4):
            d = torch.linalg.vector_norm(a[:, :, v] - b[:, :, v]).item()
            nb = torch.linalg.vector_norm(b[:, :, v]).item()
            assert d <= tol * nb, (degree, prec, (wx, wy), v, d / nb)
