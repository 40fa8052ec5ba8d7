"""Differentiable rollouts through the hand-written ADER-DG adjoint.

`Rollout` is a torch.autograd.Function whose forward advances a mesh
`nsteps` FP64 steps (adg_step) and whose backward runs the discrete adjoint
of every step in reverse (adg_step_adjoint), recomputing the states of each
checkpoint segment forward first (checkpoint every `ckpt_every` steps, so
only nsteps / ckpt_every states plus one segment are held).

Around it, for the warm-bubble sensitivity problem: the map from nodal
initial theta' to the conserved state (the bubble initialisation of
Sec. 4.2: p = pbar, T = (theta0 + theta') pi, v = 0) and the probe objective
J = sum_p (theta'(T, x_p) - target_p)^2 with theta' interpolated in the
probe's cell by the nodal Lagrange basis.  These two are small element-wise
set-up/read-out maps written with torch operations (autograd differentiates
them); the stepping and its adjoint run in libaderdg.so.
"""
import ctypes
import math

import numpy as np
import torch

from . import _lib as L


def _sp():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def step_adjoint(mesh, dt, u_n, lam_np1):
    """lam_n = (d step(u_n) / d u_n)^T lam_np1 + lam_np1 through adg_step_adjoint."""
    out = torch.empty_like(lam_np1)
    L.check(mesh._lib.adg_step_adjoint(mesh.h, float(dt), ctypes.c_void_p(u_n.data_ptr()),
                                       ctypes.c_void_p(lam_np1.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       _sp()))
    return out


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, mesh, dt, nsteps, ckpt_every):
        u0 = u0.detach().contiguous()
        ckpts = {0: u0.clone()}
        mesh.set_state(u0)
        for s in range(nsteps):
            mesh.step(dt)
            if (s + 1) % ckpt_every == 0 and s + 1 < nsteps:
                ckpts[s + 1] = mesh.get_state().clone()
        uT = mesh.get_state().clone()
        ctx.mesh, ctx.dt, ctx.nsteps, ctx.every, ctx.ckpts = mesh, dt, nsteps, ckpt_every, ckpts
        return uT

    @staticmethod
    def backward(ctx, gT):
        mesh, dt, nsteps, every = ctx.mesh, ctx.dt, ctx.nsteps, ctx.every
        lam = gT.contiguous()
        starts = list(range(0, nsteps, every))
        for s0 in reversed(starts):
            s1 = min(s0 + every, nsteps)
            states = [ctx.ckpts[s0]]
            mesh.set_state(ctx.ckpts[s0])
            for _ in range(s0, s1 - 1):
                mesh.step(dt)
                states.append(mesh.get_state().clone())
            for s in reversed(range(s0, s1)):
                lam = step_adjoint(mesh, dt, states[s - s0], lam)
        return lam, None, None, None, None


# ------------------------------------------------------------ bubble problem
def _gl(n):
    x, _ = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0)


def node_heights(cfg, device):
    n = cfg.degree + 1
    xi = torch.tensor(_gl(n), dtype=torch.float64, device=device)
    iy = torch.arange(cfg.nx * cfg.ny, device=device) // cfg.nx
    z = cfg.y0 + (iy[:, None].double() + xi[None, :]) * (cfg.Ly / cfg.ny)  # [c, j]
    return z[:, :, None].expand(-1, n, n)


def theta_to_state(theta_p, cfg):
    """Conserved state of the isentropic background (theta0, p0, g) carrying
    the temperature perturbation theta' at rest (theta_p: [c, j, i])."""
    z = node_heights(cfg, theta_p.device)
    cp = cfg.gamma * cfg.R / (cfg.gamma - 1.0)
    ex = 1.0 - cfg.g * z / (cp * cfg.theta0)
    pb = cfg.p0 * ex ** (cp / cfg.R)
    rho = pb / (cfg.R * (cfg.theta0 + theta_p) * ex)
    E = pb / (cfg.gamma - 1.0) + rho * cfg.g * z
    zero = torch.zeros_like(rho)
    return torch.stack([rho, zero, zero, E], 1).contiguous()


def state_to_theta(u, cfg):
    """theta' = T (p0/p)^(R/cp) - theta0 at the nodes."""
    z = node_heights(cfg, u.device)
    cp = cfg.gamma * cfg.R / (cfg.gamma - 1.0)
    rho, mx, my, E = u[:, 0], u[:, 1], u[:, 2], u[:, 3]
    p = (cfg.gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho - rho * cfg.g * z)
    T = p / (rho * cfg.R)
    return T * (cfg.p0 / p) ** (cfg.R / cp) - cfg.theta0


def probe_operator(cfg, probes, device):
    """(cell index, weights [P, n, n]) of Lagrange interpolation at probe points."""
    n = cfg.degree + 1
    xi = _gl(n)
    hx, hy = cfg.Lx / cfg.nx, cfg.Ly / cfg.ny
    cells, W = [], []
    for (x, y) in probes:
        ix = min(int((x - cfg.x0) / hx), cfg.nx - 1)
        iy = min(int((y - cfg.y0) / hy), cfg.ny - 1)
        sx = (x - cfg.x0) / hx - ix
        sy = (y - cfg.y0) / hy - iy
        lx = np.array([np.prod([(sx - xi[m]) / (xi[a] - xi[m]) for m in range(n) if m != a]) for a in range(n)])
        ly = np.array([np.prod([(sy - xi[m]) / (xi[a] - xi[m]) for m in range(n) if m != a]) for a in range(n)])
        cells.append(iy * cfg.nx + ix)
        W.append(np.outer(ly, lx))  # [j, i]
    return (torch.tensor(cells, device=device),
            torch.tensor(np.array(W), dtype=torch.float64, device=device))


def probe_objective(u, cfg, cells, W, target):
    th = state_to_theta(u, cfg)                       # [c, j, i]
    vals = (th[cells] * W).sum(dim=(1, 2))           # [P]
    return ((vals - target) ** 2).sum()


def objective_from_theta(theta0_p, mesh, dt, nsteps, ckpt_every, cells, W, target):
    """J(theta'_0) through the GPU rollout (differentiable)."""
    u0 = theta_to_state(theta0_p, mesh.cfg)
    uT = Rollout.apply(u0, mesh, dt, nsteps, ckpt_every)
    return probe_objective(uT, mesh.cfg, cells, W, target)
