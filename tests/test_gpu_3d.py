"""3D FP64 ADER-DG on the GPU (adg3_*) against the 3D oracle
(oracle/aderdg3d.py): relative L2 per variable <= 1e-11 (momentum floored at
|rho| * 1 m/s), as the 2D FP64 parity tests; every degree 1-4, ragged
meshes, slip walls with gravity, periodic boxes, the ABC field's analytic
boundaries, and the full 25^3 bubble mesh of the timed configuration.
The mixed-precision form (FP32 predictor on perturbations, corrector with
FP32 flux average and lifting, FP64 jumps and update)
is held to the 2D mixed path's bound: theta' relative L2 <= 1e-6."""
import math

import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.solver import Mesh3, Mesh3Config, bubble3d_config, abc_config
from oracle import physics as ph
from oracle import physics3d as p3
from oracle.aderdg3d import Mesh3 as OMesh3, Solver3

pytestmark = pytest.mark.gpu

TOL = 1e-11
BC = {L.ADG_BC_PERIODIC: "periodic", L.ADG_BC_WALL: "wall", L.ADG_BC_ANALYTIC: "dirichlet"}


def oracle3(cfg):
    P = ph.Params(N=cfg.degree, gamma=cfg.gamma, Pr=cfg.Pr, R=cfg.R, mu=cfg.mu, gravity=bool(cfg.gravity),
                  g=cfg.g, p0=cfg.p0, theta0=cfg.theta0, source="none")
    m = OMesh3(cfg.nx, cfg.ny, cfg.nz, cfg.x0, cfg.y0, cfg.z0, cfg.Lx, cfg.Ly, cfg.Lz, BC[cfg.bc_x],
               BC[cfg.bc_y], BC[cfg.bc_z], dirichlet=p3.abc_flow)
    return Solver3(m, P)


def assert_close(a, b, tol=TOL, what=""):
    a = a.detach().cpu().double()
    b = b.detach().cpu().double()
    nrho = torch.linalg.vector_norm(b[:, 0]).item()
    for v in range(5):
        d = torch.linalg.vector_norm(a[:, v] - b[:, v]).item()
        nb = torch.linalg.vector_norm(b[:, v]).item()
        den = max(nb, nrho) if v in (1, 2, 3) else nb
        assert d <= tol * den, f"{what} var {v}: rel={d / den:.3e}"


def stirred(o, seed, amp=1.0):
    """3D cosine bubble (with gravity) or a smooth density field (without),
    plus seeded smooth momentum in all three directions."""
    P = o.P
    a = inputs.smooth_perturbation((9,), seed, 1.0)
    X, Y, Z = o.X, o.Y, o.Z
    Lx, Ly, Lz = o.m.Lx, o.m.Ly, o.m.Lz
    kx, ky, kz = 2 * math.pi / Lx, 2 * math.pi / Ly, 2 * math.pi / Lz
    if P.gravity:
        th = p3.cosine_bubble(X, Y, Z)
        q = p3.bubble_state(Z, th, P)
        rho, E0 = q[0], q[4]
    else:
        rho = 1.0 + 0.2 * torch.sin(kx * X + a[0]) * torch.cos(ky * Y) * torch.sin(kz * Z + a[1])
        E0 = 2.5 + 0.1 * torch.cos(kx * X + ky * Y + kz * Z)
    u = amp * a[2] * torch.sin(ky * Y + a[3]) * torch.cos(kz * Z)
    v = amp * a[4] * torch.sin(kz * Z + a[5]) * torch.cos(kx * X)
    w = amp * a[6] * torch.cos(kx * X + a[7]) * torch.sin(ky * Y + a[8])
    E = E0 + 0.5 * rho * (u * u + v * v + w * w)
    return torch.stack([rho, rho * u, rho * v, rho * w, E], 1)


def run(cfg, u0, steps, t0=0.0, dt=None):
    o = oracle3(cfg)
    if dt is None:
        dt = 0.5 * o.stable_dt(u0, 0.5)
    m = Mesh3(cfg)
    m.set_state(u0)
    m.time = t0
    uo, t = u0, t0
    for _ in range(steps):
        uo = o.step(uo, dt, t)
        t += dt
    m.step(dt, steps)
    assert abs(m.time - t) < 1e-12
    return m.get_state(), uo


def test_init_scenarios_match_oracle():
    cfg = bubble3d_config(degree=2, n=5)
    o = oracle3(cfg)
    m = Mesh3(cfg)
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    want = torch.stack(p3.bubble_state(o.Z, p3.cosine_bubble(o.X, o.Y, o.Z), o.P), 1)
    assert_close(m.get_state(), want, 1e-14, "cosine")
    cfg = abc_config(degree=3, n=4)
    o = oracle3(cfg)
    m = Mesh3(cfg)
    m.time = 0.25
    m.init_scenario(L.ADG_SCEN_ABC)
    assert_close(m.get_state(), o.interpolate(p3.abc_flow, 0.25), 1e-14, "abc")


@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_bubble_walls_match_oracle(degree):
    """Ragged 3 x 4 x 5 mesh (not a multiple of the cells per block), slip
    walls on all sides, gravity, mu = 0.5 (viscous terms visible), the
    stirred bubble; 2 steps."""
    cfg = bubble3d_config(degree=degree, n=3, mu=0.5)
    cfg.ny, cfg.nz = 4, 5
    o = oracle3(cfg)
    a, b = run(cfg, stirred(o, degree), 2)
    assert_close(a, b, TOL, f"N={degree}")


@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_periodic_box_matches_oracle_and_conserves(degree):
    cfg = Mesh3Config(degree=degree, nx=3, ny=2, nz=4, Lx=6.0, Ly=5.0, Lz=7.0, mu=0.1)
    o = oracle3(cfg)
    u0 = stirred(o, 10 + degree)
    I0 = o.integral(u0)
    a, b = run(cfg, u0, 3)
    assert_close(a, b, TOL, f"N={degree}")
    Ia = o.integral(a.cpu())
    assert ((Ia - I0).abs() <= 1e-13 * I0.abs().clamp(min=1.0)).all(), Ia - I0


def test_mixed_boundaries_match_oracle():
    """Periodic x, walls y and z with gravity on a 5 x 2 x 3 mesh."""
    cfg = bubble3d_config(degree=2, n=5, mu=0.2)
    cfg.ny, cfg.nz, cfg.bc_x = 2, 3, L.ADG_BC_PERIODIC
    o = oracle3(cfg)
    a, b = run(cfg, stirred(o, 31), 3)
    assert_close(a, b, TOL, "mixed bc")


@pytest.mark.parametrize("degree", [2, 3])
def test_abc_analytic_boundaries_match_oracle(degree):
    cfg = abc_config(degree=degree, n=3)
    cfg.nx, cfg.nz = 4, 2
    o = oracle3(cfg)
    u0 = o.interpolate(p3.abc_flow, 0.1)
    u0 = u0 + torch.from_numpy(inputs.perturbation(tuple(u0.shape), degree, 1e-3))
    a, b = run(cfg, u0, 2, t0=0.1)
    assert_close(a, b, TOL, f"abc N={degree}")


def test_stable_dt_matches_oracle():
    cfg = bubble3d_config(degree=3, n=4)
    o = oracle3(cfg)
    u0 = stirred(o, 5)
    m = Mesh3(cfg)
    m.set_state(u0)
    want = o.stable_dt(u0, 0.5)
    assert abs(m.stable_dt(0.5) - want) <= 1e-13 * want


def test_full_size_bubble_one_step_matches_oracle():
    """The timed configuration: 25^3 cells of 40 m, degree 2, mu = 0.005,
    from the device initialisation, one step at CFL 0.5, every node compared."""
    cfg = bubble3d_config()
    o = oracle3(cfg)
    m = Mesh3(cfg)
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    u0 = m.get_state().cpu()
    dt = m.stable_dt(0.5)
    m.step(dt)
    uo = o.step(u0, dt)
    assert_close(m.get_state(), uo, TOL, "25^3")


def test_rejects_unsupported_options():
    for kw in (dict(degree=5), dict(max_levels=1), dict(source=L.ADG_SRC_STEADY)):
        cfg = bubble3d_config(degree=2, n=3)
        for k, v in kw.items():
            setattr(cfg, k, v)
        with pytest.raises(L.AdgError):
            Mesh3(cfg)
    cfg = abc_config(degree=2, n=3)
    cfg.bc_field = L.ADG_FIELD_TAYLOR_GREEN
    with pytest.raises(L.AdgError):
        Mesh3(cfg)
    cfg = abc_config(degree=2, n=3)
    cfg.gravity = 1
    with pytest.raises(L.AdgError):
        Mesh3(cfg)


# ---------------------------------------------------------------- mixed
THETA_TOL = 1e-6   # the 2D mixed path's stated bound on theta'


def rel_theta_err(o, a, b):
    w = o.b.w
    W = w[None, :, None, None] * w[None, None, :, None] * w[None, None, None, :]
    ta = p3.theta(a.unbind(1), o.Z, o.P) - o.P.theta0
    tb = p3.theta(b.unbind(1), o.Z, o.P) - o.P.theta0
    return (torch.sqrt((W * (ta - tb) ** 2).sum()) / torch.sqrt((W * tb ** 2).sum())).item()


def mixed(cfg):
    cfg.precision = L.ADG_PREC_MIXED
    return cfg


@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_mixed_bubble_every_degree(degree):
    """FP32 predictor on perturbations, FP64 corrector: ragged 3 x 4 x 5
    walled mesh, the stirred bubble, 12 steps; theta' within THETA_TOL,
    total rho within 1e-9, momentum (floored at |rho| 1 m/s) within 1e-6."""
    cfg = mixed(bubble3d_config(degree=degree, n=3, mu=0.5))
    cfg.ny, cfg.nz = 4, 5
    o = oracle3(cfg)
    a, b = run(cfg, stirred(o, 40 + degree), 12)
    a = a.cpu()
    err = rel_theta_err(o, a, b)
    assert err <= THETA_TOL, (degree, err)
    assert (torch.linalg.vector_norm(a[:, 0] - b[:, 0]) / torch.linalg.vector_norm(b[:, 0])).item() <= 1e-9
    assert_close(a, b, 1e-6, f"mixed N={degree}")


def test_mixed_full_size_bubble():
    """The timed configuration in mixed precision: 25^3, degree 2, device
    initialisation, 3 steps at the bubble CFL."""
    cfg = mixed(bubble3d_config())
    o = oracle3(cfg)
    m = Mesh3(cfg)
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    u = m.get_state().cpu()
    dt = m.stable_dt(0.25)
    m.step(dt, 3)
    for _ in range(3):
        u = o.step(u, dt)
    a = m.get_state().cpu()
    assert rel_theta_err(o, a, u) <= THETA_TOL
    assert (torch.linalg.vector_norm(a[:, 0] - u[:, 0]) / torch.linalg.vector_norm(u[:, 0])).item() <= 1e-9


def test_mixed_abc_full_state_fp32():
    """No gravity: the FP32 predictor carries the whole state; relative L2
    per variable at FP32 level (<= 1e-6) after 3 steps with analytic
    boundaries."""
    cfg = mixed(abc_config(degree=2, n=3))
    cfg.nx = 4
    o = oracle3(cfg)
    u0 = o.interpolate(p3.abc_flow, 0.1)
    a, b = run(cfg, u0, 3, t0=0.1)
    assert_close(a, b, 1e-6, "mixed abc")


@pytest.mark.parametrize("shape,bc", [((1, 1, 1), "periodic"), ((1, 2, 1), "wall"), ((2, 1, 3), "wall")])
def test_degenerate_meshes_match_oracle(shape, bc):
    """One cell per direction (a periodic cell is its own neighbour on every
    face; a walled single cell has walls on both sides), FP64 and mixed."""
    nx, ny, nz = shape
    for prec in (L.ADG_PREC_FP64, L.ADG_PREC_MIXED):
        if bc == "periodic":
            cfg = Mesh3Config(degree=2, nx=nx, ny=ny, nz=nz, Lx=6.0, Ly=5.0, Lz=7.0, mu=0.1)
        else:
            cfg = bubble3d_config(degree=2, n=1, mu=0.5)
            cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
        cfg.precision = prec
        o = oracle3(cfg)
        a, b = run(cfg, stirred(o, 50 + nx + 3 * ny + 7 * nz), 3)
        if prec == L.ADG_PREC_FP64:
            assert_close(a, b, TOL, f"{shape} {bc}")
        else:
            assert_close(a, b, 1e-6, f"{shape} {bc} mixed")
