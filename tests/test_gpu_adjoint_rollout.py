"""Gradient of a final-time potential-temperature misfit with respect to the
initial theta' DOFs through the checkpointed GPU adjoint rollout: against
central finite differences of the GPU forward rollout and against the
oracle's discrete adjoint (reverse-mode through the oracle rollout)."""
import numpy as np
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.adjoint import (objective_from_theta, probe_objective, probe_operator,
                                            state_to_theta, theta_to_state)
from paper_1905_05524_gb300.solver import Mesh, atmosphere_config
from tests.oracle_bridge import oracle_for
from oracle import physics as ph
from oracle.basis import lagrange_values

pytestmark = pytest.mark.gpu


def _setup(nx, degree=3, nprobes=64):
    cfg = atmosphere_config(degree=degree, nx=nx, ny=nx)
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    dt = m.stable_dt(0.25)
    o = oracle_for(cfg)
    th0 = ph.cosine_bubble(o.X, o.Y).cuda()                  # nodal initial theta' [c, j, i]
    probes = inputs.probes(nprobes, seed=1)
    target = torch.from_numpy(inputs.normal_values(nprobes, seed=0, scale=0.1)).cuda()
    cells, W = probe_operator(cfg, probes, "cuda")
    return cfg, m, dt, o, th0, probes, target, cells, W


def _grad(th0, m, dt, nsteps, every, cells, W, target):
    x = th0.clone().requires_grad_(True)
    J = objective_from_theta(x, m, dt, nsteps, every, cells, W, target)
    (g,) = torch.autograd.grad(J, x)
    return float(J.detach()), g


def _J(th, m, dt, nsteps, cells, W, target):
    m.set_state(theta_to_state(th, m.cfg))
    m.step(dt, nsteps)
    return float(probe_objective(m.get_state(), m.cfg, cells, W, target))


def test_rollout_gradient_vs_oracle_adjoint():
    """9x9 cells, degree 3, 10 steps (checkpoint every 4): GPU gradient equals
    the oracle's reverse-mode gradient to 1e-9 relative."""
    cfg, m, dt, o, th0, probes, target, cells, W = _setup(9, nprobes=16)
    J, g = _grad(th0, m, dt, 10, 4, cells, W, target)
    # oracle: same objective, reverse mode through its own rollout
    x = th0.cpu().clone().requires_grad_(True)
    with torch.enable_grad():
        u = torch.stack(ph.bubble_state(o.X, o.Y, x, o.P), 1)
        for _ in range(10):
            u = o.step(u, dt)
        th = ph.theta(u.unbind(1), o.Y, o.P) - o.P.theta0
        n = cfg.degree + 1
        vals = []
        for (px, py), c in zip(probes, cells.cpu().tolist()):
            ix, iy = c % cfg.nx, c // cfg.nx
            hx, hy = cfg.Lx / cfg.nx, cfg.Ly / cfg.ny
            lx = lagrange_values(o.b.xi, [px / hx - ix])[0]
            ly = lagrange_values(o.b.xi, [py / hy - iy])[0]
            vals.append((th[c] * ly[:, None] * lx[None, :]).sum())
        Jo = ((torch.stack(vals) - target.cpu()) ** 2).sum()
        (go,) = torch.autograd.grad(Jo, x)
    assert abs(J - float(Jo)) <= 1e-10 * abs(float(Jo))
    r = (torch.linalg.vector_norm(g.cpu() - go) / torch.linalg.vector_norm(go)).item()
    assert r <= 1e-9, r


def test_adjoint_run_27x27_gradient_vs_central_differences():
    """The adjoint run: degree 3, 27x27 cells, 200 steps, checkpoints every 20, 64
    probes; 32 seeded unit directions.  Step h = 1e-2 K along a unit
    direction over 11,664 DOFs: with h = 1e-6 the central difference is
    dominated by the FP64 rounding noise of J after 200 steps (~5e-14, from the
    p - pbar cancellation), which alone gives relative differences of 1e-6 to
    1e-3; at h = 1e-2 the truncation error is far below the 1e-5 bound."""
    cfg, m, dt, o, th0, probes, target, cells, W = _setup(27)
    J, g = _grad(th0, m, dt, 200, 20, cells, W, target)
    dirs = inputs.directions(32, th0.numel(), seed=2)
    h = 1e-2
    worst = 0.0
    for d_np in dirs:
        d = torch.from_numpy(d_np).reshape(th0.shape).cuda()
        fd = (_J(th0 + h * d, m, dt, 200, cells, W, target) - _J(th0 - h * d, m, dt, 200, cells, W, target)) / (2 * h)
        ad = float((g * d).sum())
        worst = max(worst, abs(fd - ad) / max(abs(ad), 1e-300))
    print(f"adjoint run: J = {J:.6e}, worst relative FD error over 32 directions = {worst:.3e}")
    assert worst <= 1e-5, worst
