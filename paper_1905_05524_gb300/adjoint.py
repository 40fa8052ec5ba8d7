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
probe's cell by the nodal Lagrange basis.  Both maps and their adjoints run
in libaderdg.so too (adg_theta_to_state, adg_theta_to_state_adjoint,
adg_probe_objective); the autograd Functions below only pass device arrays.
"""
import ctypes

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
class ThetaToState(torch.autograd.Function):
    """u = state(theta') (adg_theta_to_state); backward: adg_theta_to_state_adjoint."""

    @staticmethod
    def forward(ctx, theta_p, mesh):
        th = theta_p.detach().contiguous()
        n = mesh.cfg.degree + 1
        u = torch.empty(th.shape[0], 4, n, n, dtype=torch.float64, device=th.device)
        L.check(mesh._lib.adg_theta_to_state(mesh.h, ctypes.c_void_p(th.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                             _sp()))
        ctx.mesh = mesh
        ctx.save_for_backward(th)
        return u

    @staticmethod
    def backward(ctx, lam_u):
        (th,) = ctx.saved_tensors
        lam_u = lam_u.contiguous()
        out = torch.empty_like(th)
        L.check(ctx.mesh._lib.adg_theta_to_state_adjoint(ctx.mesh.h, ctypes.c_void_p(th.data_ptr()),
                                                         ctypes.c_void_p(lam_u.data_ptr()),
                                                         ctypes.c_void_p(out.data_ptr()), _sp()))
        return out, None


class ProbeObjective(torch.autograd.Function):
    """J(u) = sum_p (theta'(u; x_p) - target_p)^2 (adg_probe_objective, which
    also returns dJ/du for the backward)."""

    @staticmethod
    def forward(ctx, u, mesh, probes_xy, target):
        u = u.detach().contiguous()
        xy = probes_xy.contiguous()
        tg = target.contiguous()
        resid = torch.empty_like(tg)
        J = torch.empty((), dtype=torch.float64, device=u.device)
        g = torch.empty_like(u)
        L.check(mesh._lib.adg_probe_objective(mesh.h, ctypes.c_void_p(u.data_ptr()), int(tg.numel()),
                                              ctypes.c_void_p(xy.data_ptr()), ctypes.c_void_p(tg.data_ptr()),
                                              ctypes.c_void_p(resid.data_ptr()), ctypes.c_void_p(J.data_ptr()),
                                              ctypes.c_void_p(g.data_ptr()), _sp()))
        ctx.save_for_backward(g)
        return J

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ * g, None, None, None


def theta_to_state(theta_p, mesh):
    """Conserved state of the isentropic background carrying theta' at rest."""
    return ThetaToState.apply(theta_p, mesh)


def state_to_theta(u, mesh):
    """theta' = T (p0/p)^(R/cp) - theta0 at the nodes (adg_state_to_theta)."""
    u = u.detach().contiguous()
    n = mesh.cfg.degree + 1
    th = torch.empty(u.shape[0], n, n, dtype=torch.float64, device=u.device)
    L.check(mesh._lib.adg_state_to_theta(mesh.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(th.data_ptr()),
                                         _sp()))
    return th


def probe_objective(u, mesh, probes_xy, target):
    return ProbeObjective.apply(u, mesh, probes_xy, target)


def objective_from_theta(theta0_p, mesh, dt, nsteps, ckpt_every, probes_xy, target):
    """J(theta'_0) through the GPU rollout (differentiable)."""
    u0 = theta_to_state(theta0_p, mesh)
    uT = Rollout.apply(u0, mesh, dt, nsteps, ckpt_every)
    return probe_objective(uT, mesh, probes_xy, target)
