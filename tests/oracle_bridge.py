"""Builds the oracle solver that matches a MeshConfig (test infrastructure).

Only translates descriptor fields into oracle.Mesh / oracle.physics.Params;
no arithmetic of the method lives here.
"""
from oracle.aderdg import Mesh as OMesh, Solver as OSolver
from oracle import physics as ph


def oracle_for(cfg):
    bc = {0: "periodic", 1: "wall", 5: "noslip", 6: "dirichlet"}
    field = {0: None, 1: ph.taylor_green}[getattr(cfg, "bc_field", 0)]
    mesh = OMesh(nx=cfg.nx, ny=cfg.ny, x0=cfg.x0, y0=cfg.y0, Lx=cfg.Lx, Ly=cfg.Ly,
                 bc_x=bc[cfg.bc_x], bc_y=bc[cfg.bc_y], lid_u=getattr(cfg, "lid_u", 0.0), dirichlet=field)
    P = ph.Params(N=cfg.degree, gamma=cfg.gamma, Pr=cfg.Pr, R=cfg.R, mu=cfg.mu,
                  gravity=bool(cfg.gravity), g=cfg.g, p0=cfg.p0, theta0=cfg.theta0,
                  source={0: "none", 1: "steady", 2: "paper"}[cfg.source])
    return OSolver(mesh, P)


def steady_field(solver, cfg):
    """Oracle nodal interpolation of the steady manufactured field of cfg."""
    import functools
    fn = functools.partial(ph.steady_manufactured, a=cfg.src_a, L=cfg.src_L, U=cfg.src_U, p=cfg.src_p)
    return solver.interpolate(lambda x, y, t, P: fn(x, y, t, P))


def paper_field(solver, t=0.0):
    """Oracle nodal interpolation of the Eq. 8 field at time t."""
    return solver.interpolate(ph.paper_manufactured, t)


def taylor_green_field(solver, t=0.0):
    """Oracle nodal interpolation of the Taylor-Green field at time t."""
    return solver.interpolate(ph.taylor_green, t)


def cavity_field(solver):
    """Fluid at rest, rho = 1, p = 100/gamma."""
    import torch
    P = solver.P
    one = torch.ones_like(solver.X)
    return torch.stack([one, 0.0 * one, 0.0 * one, (100.0 / P.gamma) / (P.gamma - 1.0) * one], 1)


def cosine_field(solver, A=0.5, a=250.0, xc=500.0, zc=350.0):
    import torch
    th = ph.cosine_bubble(solver.X, solver.Y, A, a, xc, zc)
    return torch.stack(ph.bubble_state(solver.X, solver.Y, th, solver.P), 1)


def two_bubble_field(solver):
    import torch
    th = ph.two_bubbles(solver.X, solver.Y)
    return torch.stack(ph.bubble_state(solver.X, solver.Y, th, solver.P), 1)


def background_field(solver):
    import torch
    th = 0.0 * solver.X
    return torch.stack(ph.bubble_state(solver.X, solver.Y, th, solver.P), 1)
