"""Local time stepping across the levels of an adaptive mesh on the GPU
(adg_step_lts) against the oracle's step_lts (reading L1): periodic trees
of two and three levels, the walled bubble with hanging faces and gravity,
one level (equal to the global step), and conservation over cycles."""
import math

import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.solver import Mesh, MeshConfig, atmosphere_config
from oracle.amr import AmrSolver
from oracle import physics as ph
from tests.tolerances import momentum_floor

pytestmark = pytest.mark.gpu


def _wave(X, Y, P):
    rho = 1.0 + 0.2 * torch.sin(2 * math.pi * (X + Y) / 6.0)
    return [rho, rho * 1.0, rho * 0.5, 1.0 / (P.gamma - 1) + 0.5 * rho * 1.25]


def _close(a, b, tol=1e-11, floor=0.0):
    for v in range(4):
        d = torch.linalg.vector_norm(a[:, v] - b[:, v]).item()
        nb = torch.linalg.vector_norm(b[:, v]).item()
        bound = tol * nb + (floor if v in (1, 2) else 0.0)
        assert d <= bound, (v, d, nb, bound)


def _periodic_tree(degree, levels, seed=1, frac=0.3):
    cfg = MeshConfig(degree=degree, nx=6, ny=6, Lx=6.0, Ly=6.0, mu=0.05, max_levels=levels)
    P = ph.Params(N=degree, gamma=cfg.gamma, Pr=cfg.Pr, R=cfg.R, mu=cfg.mu, gravity=False, source="none")
    o = AmrSolver(6, 6, P, 6.0, 6.0, bc="periodic", max_level=levels)
    m = Mesh(cfg)
    u = o.interpolate_field(lambda X, Y: _wave(X, Y, P))
    for lv in range(levels):
        fl = (torch.from_numpy(inputs.uniform_values(len(o.leaves), seed=seed + lv, lo=0, hi=1)) < frac).to(torch.int8)
        u = o.adapt(u, fl)
        m.adapt(fl.cuda())
    assert m.leaf_info() == [tuple(c) for c in o.leaves]
    u = u + torch.from_numpy(inputs.perturbation(tuple(u.shape), seed=7, scale=0.01))
    m.set_state(u.cuda().contiguous())
    return m, o, u


@pytest.mark.parametrize("degree,levels", [(2, 1), (3, 1), (5, 1), (3, 2)])
def test_lts_periodic_tree_matches_oracle(degree, levels):
    m, o, u = _periodic_tree(degree, levels)
    assert len(o.levels()) == levels + 1
    dt = 0.0015 / 3 ** (levels - 1)
    uo, T = o.step_lts(u, dt)
    c = m.step_lts(dt)
    assert abs(c - T) <= 1e-15 * T
    _close(m.get_state().cpu(), uo)
    m.close()


@pytest.mark.parametrize("degree", [3, 5])
def test_lts_bubble_walls_hanging_faces_matches_oracle(degree):
    """Cosine bubble with slip walls, gravity and a refined patch on a 6x6
    base: one cycle (3 fine steps) against the oracle; the momentum floor of
    the fine cells for the background rounding."""
    cfg = atmosphere_config(degree=degree, nx=6, ny=6)
    cfg.max_levels = 1
    P = ph.Params(N=degree, gamma=cfg.gamma, Pr=cfg.Pr, R=cfg.R, mu=cfg.mu, gravity=True, g=cfg.g, p0=cfg.p0,
                  theta0=cfg.theta0, source="none")
    o = AmrSolver(6, 6, P, 1000.0, 1000.0, bc="wall", max_level=1)
    m = Mesh(cfg)
    X, Y = o.node_coords()
    u = torch.stack(ph.bubble_state(X, Y, ph.cosine_bubble(X, Y), P), 1)
    fl = torch.zeros(36, dtype=torch.int8)
    fl[[13, 14, 15, 20, 21, 28]] = 1
    u = o.adapt(u, fl)
    m.adapt(fl.cuda())
    m.set_state(u.cuda().contiguous())
    dt = m.stable_dt(0.25)
    uo, T = o.step_lts(u, dt)
    c = m.step_lts(dt)
    assert abs(c - 3 * dt) <= 1e-15 * c
    fine = atmosphere_config(degree=degree, nx=18, ny=18)
    _close(m.get_state().cpu(), uo, floor=momentum_floor(fine, dt, 3, u[:, 0].numel()))
    m.close()


def test_lts_single_level_equals_global_step():
    cfg = MeshConfig(degree=3, nx=5, ny=4, Lx=6.0, Ly=6.0, mu=0.05, max_levels=1)
    P = ph.Params(N=3, gamma=cfg.gamma, Pr=cfg.Pr, R=cfg.R, mu=cfg.mu, gravity=False, source="none")
    o = AmrSolver(5, 4, P, 6.0, 6.0, bc="periodic", max_level=1)
    u = o.interpolate_field(lambda X, Y: _wave(X, Y, P))
    a, b = Mesh(cfg), Mesh(cfg)
    a.set_state(u.cuda().contiguous())
    b.set_state(u.cuda().contiguous())
    assert a.step_lts(0.004) == 0.004
    b.step(0.004)
    ua, ub = a.get_state(), b.get_state()
    assert (ua - ub).abs().max().item() <= 1e-14 * ub.abs().max().item()
    a.close()
    b.close()


def test_lts_conserves_on_gpu():
    m, o, u = _periodic_tree(3, 2)
    I0 = o.integral(u)
    for _ in range(3):
        m.step_lts(0.0002)   # CFL ~0.3 on the finest leaves (viscous limit)
    I1 = o.integral(m.get_state().cpu())
    assert ((I1 - I0).abs() <= 1e-13 * I0.abs().clamp(min=1.0)).all(), (I1 - I0)
    m.close()


def test_lts_refuses_uniform_and_mixed():
    m = Mesh(MeshConfig(degree=3, nx=4, ny=4, Lx=6.0, Ly=6.0))
    with pytest.raises(L.AdgError) as e:
        m.step_lts(0.001)
    assert e.value.code == L.ADG_EINVAL
    cfg = atmosphere_config(degree=3, nx=6, ny=6, precision=L.ADG_PREC_MIXED)
    cfg.max_levels = 1
    m2 = Mesh(cfg)
    with pytest.raises(L.AdgError) as e:
        m2.step_lts(0.001)
    assert e.value.code == L.ADG_EUNSUPPORTED
