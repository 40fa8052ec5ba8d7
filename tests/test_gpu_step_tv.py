"""adg_step_tv (step with the TV indicator evaluated in the corrector's
epilogue) gives bitwise the results of adg_step followed by
adg_tv_indicator: state, per-cell TV, flags, mean and sigma; FP64 and mixed
forms, theta and rho indicators, ragged tiles, adaptive meshes."""
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.solver import Mesh, atmosphere_config, steady_manufactured_config

pytestmark = pytest.mark.gpu


def pair(cfg, init, var, T_r, T_c, steps=3):
    a, b = Mesh(cfg), Mesh(cfg)
    init(a)
    init(b)
    dt = a.stable_dt(0.25)
    for _ in range(steps):
        a.step(dt)
        ta, fa, sa = a.tv_indicator(var, T_r, T_c)
        tb, fb, sb = b.step_tv(dt, var, T_r, T_c)
    torch.cuda.synchronize()
    assert torch.equal(a.get_state(), b.get_state())
    assert torch.equal(ta, tb)
    assert torch.equal(fa, fb)
    assert sa == sb
    assert a.time == b.time
    return tb, fb


def bubble(m):
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)


@pytest.mark.parametrize("prec", [L.ADG_PREC_FP64, L.ADG_PREC_MIXED])
@pytest.mark.parametrize("degree,nx,ny", [(3, 11, 9), (5, 13, 7)])
def test_step_tv_bubble_theta(prec, degree, nx, ny):
    tv, fl = pair(atmosphere_config(degree=degree, nx=nx, ny=ny, precision=prec), bubble, L.ADG_TV_THETA, 1.5, -0.5)
    assert (tv > 0).any() and (fl == 1).any()


@pytest.mark.parametrize("prec", [L.ADG_PREC_FP64, L.ADG_PREC_MIXED])
def test_step_tv_bubble_rho(prec):
    pair(atmosphere_config(degree=4, nx=9, ny=10, precision=prec), bubble, L.ADG_TV_RHO, 1.0, -0.5)


def test_step_tv_steady_rho_fp64():
    def init(m):
        m.init_scenario(L.ADG_SCEN_STEADY)
        u = m.get_state()
        m.set_state(u + torch.from_numpy(inputs.perturbation(tuple(u.shape), seed=11, scale=1e-3)).to(u.device))
    pair(steady_manufactured_config(degree=2, nx=7, ny=5), init, L.ADG_TV_RHO, 1.0, -0.5)


def test_step_tv_adaptive_mesh():
    cfg = atmosphere_config(degree=2, nx=9, ny=9)
    cfg.max_levels = 1
    pair(cfg, bubble, L.ADG_TV_THETA, 1.5, -0.5, steps=2)
