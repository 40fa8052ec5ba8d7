"""Gradient of a final-time potential-temperature misfit with respect to the
initial theta' DOFs through the checkpointed GPU adjoint rollout: against
central finite differences of the GPU forward rollout and against the
oracle's discrete adjoint (reverse-mode through the oracle rollout).  The
theta' -> state map, the probe objective and their adjoints run in the
library (adg_theta_to_state, adg_theta_to_state_adjoint, adg_state_to_theta,
adg_probe_objective); they are checked here against the oracle's bubble
state and potential temperature."""
import numpy as np
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.adjoint import (objective_from_theta, probe_objective, state_to_theta,
                                            theta_to_state)
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
    xy = torch.from_numpy(probes).cuda()
    return cfg, m, dt, o, th0, probes, target, xy


def _grad(th0, m, dt, nsteps, every, xy, target):
    x = th0.clone().requires_grad_(True)
    J = objective_from_theta(x, m, dt, nsteps, every, xy, target)
    (g,) = torch.autograd.grad(J, x)
    return float(J.detach()), g


def _J(th, m, dt, nsteps, xy, target):
    m.set_state(theta_to_state(th, m))
    m.step(dt, nsteps)
    return float(probe_objective(m.get_state(), m, xy, target))


def _oracle_J(o, cfg, u, probes, target):
    """The probe objective written with the oracle's theta and Lagrange basis."""
    th = ph.theta(u.unbind(1), o.Y, o.P) - o.P.theta0
    hx, hy = cfg.Lx / cfg.nx, cfg.Ly / cfg.ny
    vals = []
    for (px, py) in probes:
        ix = min(int(px / hx), cfg.nx - 1)
        iy = min(int(py / hy), cfg.ny - 1)
        lx = lagrange_values(o.b.xi, [px / hx - ix])[0]
        ly = lagrange_values(o.b.xi, [py / hy - iy])[0]
        vals.append((th[iy * cfg.nx + ix] * ly[:, None] * lx[None, :]).sum())
    return ((torch.stack(vals) - target.cpu()) ** 2).sum()


def test_theta_maps_match_oracle():
    """theta' -> state equals the oracle's bubble state; state -> theta'
    equals the oracle's theta - theta0 (on a stirred state); the adjoint of
    theta' -> state passes the dot-product test against the oracle's
    reverse mode; and with the cosine theta' the map reproduces
    adg_init_scenario."""
    cfg, m, dt, o, th0, probes, target, xy = _setup(9, degree=4)
    u = theta_to_state(th0, m)
    uo = torch.stack(ph.bubble_state(o.X, o.Y, th0.cpu(), o.P), 1)
    assert (u.cpu() - uo).abs().max().item() <= 1e-14 * uo.abs().max().item()
    assert (u - m.get_state()).abs().max().item() <= 1e-12 * uo.abs().max().item()
    us = u.clone()
    us[:, 1:3] = torch.from_numpy(inputs.perturbation(tuple(us[:, 1:3].shape), seed=3, scale=0.5)).cuda()
    th = state_to_theta(us, m)
    tho = ph.theta(us.cpu().unbind(1), o.Y, o.P) - o.P.theta0
    assert (th.cpu() - tho).abs().max().item() <= 1e-12 * 300.0
    lam = torch.from_numpy(inputs.perturbation(tuple(u.shape), seed=4, scale=1.0)).cuda()
    x = th0.cpu().clone().requires_grad_(True)
    with torch.enable_grad():
        uo = torch.stack(ph.bubble_state(o.X, o.Y, x, o.P), 1)
        (go,) = torch.autograd.grad((uo * lam.cpu()).sum(), x)
    xg = th0.clone().requires_grad_(True)
    (gg,) = torch.autograd.grad((theta_to_state(xg, m) * lam).sum(), xg)
    assert (torch.linalg.vector_norm(gg.cpu() - go) / torch.linalg.vector_norm(go)).item() <= 1e-13
    m.close()


def test_probe_objective_and_gradient_match_oracle():
    """J and dJ/du of adg_probe_objective against the oracle's objective and
    its reverse-mode gradient on a stirred bubble state."""
    cfg, m, dt, o, th0, probes, target, xy = _setup(9, nprobes=40)
    u = theta_to_state(th0, m).clone()
    u[:, 1:3] = torch.from_numpy(inputs.perturbation(tuple(u[:, 1:3].shape), seed=5, scale=0.5)).cuda()
    x = u.cpu().clone().requires_grad_(True)
    with torch.enable_grad():
        Jo = _oracle_J(o, cfg, x, probes, target)
        (go,) = torch.autograd.grad(Jo, x)
    ug = u.clone().requires_grad_(True)
    J = probe_objective(ug, m, xy, target)
    (g,) = torch.autograd.grad(J, ug)
    Jo = float(Jo.detach())
    assert abs(float(J.detach()) - Jo) <= 1e-12 * abs(Jo)
    assert (torch.linalg.vector_norm(g.cpu() - go) / torch.linalg.vector_norm(go)).item() <= 1e-12
    m.close()


def test_rollout_gradient_vs_oracle_adjoint():
    """9x9 cells, degree 3, 10 steps (checkpoint every 4): GPU gradient equals
    the oracle's reverse-mode gradient to 1e-9 relative."""
    cfg, m, dt, o, th0, probes, target, xy = _setup(9, nprobes=16)
    J, g = _grad(th0, m, dt, 10, 4, xy, target)
    # oracle: same objective, reverse mode through its own rollout
    x = th0.cpu().clone().requires_grad_(True)
    with torch.enable_grad():
        u = torch.stack(ph.bubble_state(o.X, o.Y, x, o.P), 1)
        for _ in range(10):
            u = o.step(u, dt)
        Jo = _oracle_J(o, cfg, u, probes, target)
        (go,) = torch.autograd.grad(Jo, x)
    Jo = float(Jo.detach())
    assert abs(J - Jo) <= 1e-10 * abs(Jo)
    r = (torch.linalg.vector_norm(g.cpu() - go) / torch.linalg.vector_norm(go)).item()
    assert r <= 1e-9, r


def test_adjoint_run_27x27_gradient_vs_central_differences():
    """The adjoint run: degree 3, 27x27 cells, 200 steps, checkpoints every 20, 64
    probes; 32 seeded unit directions.  Step h = 1e-2 K along a unit
    direction over 11,664 DOFs: with h = 1e-6 the central difference is
    dominated by the FP64 rounding noise of J after 200 steps (~5e-14, from the
    p - pbar cancellation), which alone gives relative differences of 1e-6 to
    1e-3; at h = 1e-2 the truncation error is far below the 1e-5 bound."""
    cfg, m, dt, o, th0, probes, target, xy = _setup(27)
    J, g = _grad(th0, m, dt, 200, 20, xy, target)
    dirs = inputs.directions(32, th0.numel(), seed=2)
    h = 1e-2
    worst = 0.0
    for d_np in dirs:
        d = torch.from_numpy(d_np).reshape(th0.shape).cuda()
        fd = (_J(th0 + h * d, m, dt, 200, xy, target) - _J(th0 - h * d, m, dt, 200, xy, target)) / (2 * h)
        ad = float((g * d).sum())
        worst = max(worst, abs(fd - ad) / max(abs(ad), 1e-300))
    print(f"adjoint run: J = {J:.6e}, worst relative FD error over 32 directions = {worst:.3e}")
    assert worst <= 1e-5, worst
