"""Adaptive 3:1 tree on the GPU against the oracle's tree (oracle/amr.py):
identical leaf sets after adaptation, transferred states, steps across
hanging faces, conservation, TV indicator and the two-bubble run's initial-mesh
procedure (init -> TV -> refine, twice, re-initialising from the analytic
two-bubble field)."""
import math

import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from tests.tolerances import momentum_floor
from paper_1905_05524_gb300.solver import Mesh, MeshConfig, atmosphere_config
from oracle.amr import AmrSolver
from oracle import indicator as oind
from oracle import physics as ph

pytestmark = pytest.mark.gpu


def _pair(cfg, bc):
    P = ph.Params(N=cfg.degree, gamma=cfg.gamma, Pr=cfg.Pr, R=cfg.R, mu=cfg.mu, gravity=bool(cfg.gravity),
                  g=cfg.g, p0=cfg.p0, theta0=cfg.theta0, source="none")
    o = AmrSolver(cfg.nx, cfg.ny, P, cfg.Lx, cfg.Ly, cfg.x0, cfg.y0, bc=bc, max_level=cfg.max_levels)
    return Mesh(cfg), o


def _flags(k, seed, frac):
    x = torch.from_numpy(inputs.uniform_values(k, seed=seed, lo=0.0, hi=1.0))
    return torch.where(x < frac, 1, torch.where(x > 1 - frac / 2, -1, 0)).to(torch.int8)


def _close(a, b, tol=1e-11, floor=0.0):
    """Per-variable L2 |a - b| <= tol |b|, plus the momentum rounding floor
    of tests/tolerances.py (absolute) for the momentum components."""
    for v in range(4):
        d = torch.linalg.vector_norm(a[:, v] - b[:, v]).item()
        nb = torch.linalg.vector_norm(b[:, v]).item()
        bound = tol * nb + (floor if v in (1, 2) else 0.0)
        assert d <= bound, (v, d, nb, bound)


def _wave(X, Y, P):
    rho = 1.0 + 0.2 * torch.sin(2 * math.pi * (X + Y) / 6.0)
    return [rho, rho * 1.0, rho * 0.5, 1.0 / (P.gamma - 1) + 0.5 * rho * 1.25]


def test_adapt_and_step_periodic_matches_oracle():
    cfg = MeshConfig(degree=3, nx=6, ny=6, Lx=6.0, Ly=6.0, mu=0.05, max_levels=2)
    m, o = _pair(cfg, "periodic")
    u = o.interpolate_field(lambda X, Y: _wave(X, Y, o.P))
    m.set_state(u.cuda().contiguous())
    for seed, frac in ((1, 0.3), (2, 0.2), (3, 0.2)):
        fl = _flags(len(o.leaves), seed, frac)
        u = o.adapt(u, fl)
        m.adapt(fl.cuda())
        assert m.leaf_info() == [tuple(c) for c in o.leaves]
        _close(m.get_state().cpu(), u, 1e-13)
    assert len({c[0] for c in o.leaves}) >= 2
    I0 = o.integral(u)
    dt = 0.003
    for _ in range(3):
        u = o.step(u, dt)
    m.step(dt, 3)
    a = m.get_state().cpu()
    _close(a, u)
    # conservation of the GPU run on the periodic tree
    Ia = o.integral(a)
    assert ((Ia - I0).abs() <= 1e-13 * I0.abs().clamp(min=1.0)).all(), Ia - I0


@pytest.mark.parametrize("degree", [1, 2, 3, 4, 5, 6, 7])
def test_bubble_walls_hanging_faces_matches_oracle(degree):
    """Cosine bubble with slip walls on a 6x6 base with a refined patch (hanging
    faces, gravity): adaptation and 3 steps match the oracle."""
    cfg = atmosphere_config(degree=degree, nx=6, ny=6)
    cfg.max_levels = 1
    m, o = _pair(cfg, "wall")
    X, Y = o.node_coords()
    u = torch.stack(ph.bubble_state(X, Y, ph.cosine_bubble(X, Y), o.P), 1)
    m.set_state(u.cuda().contiguous())
    fl = torch.zeros(36, dtype=torch.int8)
    fl[[13, 14, 15, 20, 21, 28]] = 1
    u = o.adapt(u, fl)
    m.adapt(fl.cuda())
    assert m.leaf_info() == [tuple(c) for c in o.leaves]
    _close(m.get_state().cpu(), u, 1e-13)
    dt = m.stable_dt(0.25)
    for _ in range(3):
        u = o.step(u, dt)
    m.step(dt, 3)
    fine = atmosphere_config(degree=degree, nx=6 * 3, ny=6 * 3)  # level-1 leaves set the floor's cell size
    _close(m.get_state().cpu(), u, floor=momentum_floor(fine, dt, 3, u[:, 0].numel()))


def _oracle_tv(o, u, var):
    tv = torch.empty(len(o.leaves), dtype=torch.float64)
    for lv, idx, view in o.level_views():
        f = oind.indicator_field(view, u[idx], var)
        tv[idx] = oind.total_variation(view, f)
    return tv


def test_two_bubble_initial_mesh_and_tv_match_oracle():
    """Two-bubble field, base 27x27 on [0,1000]^2, 2 levels, T_r = 2.5,
    T_c = -0.5: init -> TV -> refine twice (refine only), re-initialising from
    the analytic field; identical leaves and TV values."""
    cfg = atmosphere_config(degree=5, nx=27, ny=27, mu=0.001)
    cfg.max_levels = 2
    m, o = _pair(cfg, "wall")
    for _ in range(2):
        X, Y = o.node_coords()
        u = torch.stack(ph.bubble_state(X, Y, ph.two_bubbles(X, Y), o.P), 1)
        m.init_scenario(L.ADG_SCEN_TWO_BUBBLES)
        _close(m.get_state().cpu(), u, 1e-13)
        tv_o = _oracle_tv(o, u, "theta")
        mean, std = oind.mean_std(tv_o)
        fl_o = oind.flags(tv_o, mean, std, 2.5, -0.5)
        tv_g, fl_g, (mg, sg) = m.tv_indicator(L.ADG_TV_THETA, 2.5, -0.5)
        floor = 1e-10 * tv_o.abs().max()
        assert bool(((tv_g.cpu() - tv_o).abs() <= 1e-11 * tv_o.abs() + floor).all())
        fl_o = torch.where(fl_o > 0, 1, 0).to(torch.int8)   # refine only while building the initial mesh
        fl_g = torch.where(fl_g > 0, 1, 0).to(torch.int8)
        assert torch.equal(fl_g.cpu(), fl_o)
        o.adapt(u, fl_o)
        m.adapt(fl_g)
        assert m.leaf_info() == [tuple(c) for c in o.leaves]
    levels = [c[0] for c in o.leaves]
    assert max(levels) >= 1 and len(levels) < 243 * 243
    print(f"two-bubble initial mesh: {len(levels)} leaves "
          f"({levels.count(0)}/{levels.count(1)}/{levels.count(2)} per level)")


# ---------------------------------------------------------------- mixed precision
THETA_TOL = 1e-6  # the mixed path's stated bound on theta' (relative L2)


def _theta_err(o, a, b):
    X, Y = o.node_coords()
    ta = ph.theta(a.unbind(1), Y, o.P) - o.P.theta0
    tb = ph.theta(b.unbind(1), Y, o.P) - o.P.theta0
    return (torch.linalg.vector_norm(ta - tb) / torch.linalg.vector_norm(tb)).item()


@pytest.mark.parametrize("degree", [1, 2, 3, 5, 7])
def test_mixed_bubble_walls_hanging_faces_matches_oracle(degree):
    """Mixed precision (FP32 predictor on perturbations, FP64 corrector) on
    the refined-patch bubble mesh with hanging faces and gravity: 6 steps
    against the FP64 oracle, theta' within THETA_TOL, total rho within
    1e-9."""
    cfg = atmosphere_config(degree=degree, nx=6, ny=6, precision=L.ADG_PREC_MIXED)
    cfg.max_levels = 1
    m, o = _pair(cfg, "wall")
    X, Y = o.node_coords()
    u = torch.stack(ph.bubble_state(X, Y, ph.cosine_bubble(X, Y), o.P), 1)
    m.set_state(u.cuda().contiguous())
    fl = torch.zeros(36, dtype=torch.int8)
    fl[[13, 14, 15, 20, 21, 28]] = 1
    u = o.adapt(u, fl)
    m.adapt(fl.cuda())
    assert m.leaf_info() == [tuple(c) for c in o.leaves]
    dt = m.stable_dt(0.25)
    for _ in range(6):
        u = o.step(u, dt)
    m.step(dt, 6)
    a = m.get_state().cpu()
    err = _theta_err(o, a, u)
    assert err <= THETA_TOL, (degree, err)
    assert (torch.linalg.vector_norm(a[:, 0] - u[:, 0]) / torch.linalg.vector_norm(u[:, 0])).item() <= 1e-9


def test_mixed_adapt_step_periodic_matches_oracle():
    """Periodic tree without gravity (the FP32 predictor carries the whole
    state), three adaptations then 3 steps at the stable dt (CFL 0.25 on the
    finest leaves; the FP64 test's fixed dt = 0.003 is ~16x above it there,
    and its unstable modes amplify FP32 rounding from step to step):
    FP32-level agreement (<= 1e-6 per variable) and conservation to 1e-8:
    the face fluxes are FP64 and shared by both sides, but the volume
    residual's cell integral, zero in exact arithmetic, carries the FP32
    rounding of its terms (about 1e-9 relative over the 3 steps)."""
    cfg = MeshConfig(degree=3, nx=6, ny=6, Lx=6.0, Ly=6.0, mu=0.05, max_levels=2, precision=L.ADG_PREC_MIXED)
    m, o = _pair(cfg, "periodic")
    u = o.interpolate_field(lambda X, Y: _wave(X, Y, o.P))
    m.set_state(u.cuda().contiguous())
    for seed, frac in ((1, 0.3), (2, 0.2), (3, 0.2)):
        fl = _flags(len(o.leaves), seed, frac)
        u = o.adapt(u, fl)
        m.adapt(fl.cuda())
        assert m.leaf_info() == [tuple(c) for c in o.leaves]
    I0 = o.integral(u)
    dt = m.stable_dt(0.25)
    for _ in range(3):
        u = o.step(u, dt)
    m.step(dt, 3)
    a = m.get_state().cpu()
    _close(a, u, 1e-6)
    Ia = o.integral(a)
    assert ((Ia - I0).abs() <= 1e-8 * I0.abs().clamp(min=1.0)).all(), Ia - I0


def test_mixed_two_bubble_run_tracks_fp64():
    """The two-bubble AMR procedure (two bubbles, 27x27 base, two levels, initial
    mesh by init -> TV -> refine twice) with an FP64 and a mixed mesh in
    lockstep -- both adapted with the FP64 mesh's flags -- then 10 steps, a
    regrid, 10 steps: theta' of the mixed run within THETA_TOL of the FP64
    run on the same leaves."""
    ms = []
    for prec in (L.ADG_PREC_FP64, L.ADG_PREC_MIXED):
        cfg = atmosphere_config(degree=5, nx=27, ny=27, mu=0.001, precision=prec)
        cfg.max_levels = 2
        ms.append(Mesh(cfg))
    for _ in range(2):
        for m in ms:
            m.init_scenario(L.ADG_SCEN_TWO_BUBBLES)
        _, fl, _ = ms[0].tv_indicator(L.ADG_TV_THETA, 2.5, -0.5)
        fl = torch.where(fl > 0, 1, 0).to(torch.int8)
        for m in ms:
            m.adapt(fl)
    for m in ms:
        m.init_scenario(L.ADG_SCEN_TWO_BUBBLES)
    dt = ms[0].stable_dt(0.25)
    for m in ms:
        m.step(dt, 10)
    _, fl, _ = ms[0].tv_indicator(L.ADG_TV_THETA, 2.5, -0.5)
    for m in ms:
        m.adapt(fl)
        m.step(dt, 10)
    assert ms[0].leaf_info() == ms[1].leaf_info()
    assert len({c[0] for c in ms[0].leaf_info()}) >= 2
    P = ph.atmosphere_params(5, mu=0.001)
    o = AmrSolver(27, 27, P, 1000.0, 1000.0, bc="wall", max_level=2)
    o.leaves = [tuple(c) for c in ms[0].leaf_info()]
    o._index()
    err = _theta_err(o, ms[1].get_state().cpu(), ms[0].get_state().cpu())
    assert err <= THETA_TOL, err


@pytest.mark.parametrize("prec", [L.ADG_PREC_FP64, L.ADG_PREC_MIXED])
def test_two_bubble_mesh_step_matches_oracle(prec):
    """A step on the full two-bubble adaptive mesh (27x27 base, two levels,
    built by init -> TV -> refine twice) against the oracle's tree: FP64 at
    1e-11, mixed within THETA_TOL of theta' and 1e-9 of rho."""
    cfg = atmosphere_config(degree=5, nx=27, ny=27, mu=0.001, precision=prec)
    cfg.max_levels = 2
    m, o = _pair(cfg, "wall")
    for _ in range(2):
        X, Y = o.node_coords()
        u = torch.stack(ph.bubble_state(X, Y, ph.two_bubbles(X, Y), o.P), 1)
        m.init_scenario(L.ADG_SCEN_TWO_BUBBLES)
        _, fl, _ = m.tv_indicator(L.ADG_TV_THETA, 2.5, -0.5)
        fl = torch.where(fl > 0, 1, 0).to(torch.int8)
        o.adapt(u, fl.cpu())
        m.adapt(fl)
    assert m.leaf_info() == [tuple(c) for c in o.leaves]
    X, Y = o.node_coords()
    u = torch.stack(ph.bubble_state(X, Y, ph.two_bubbles(X, Y), o.P), 1)
    m.init_scenario(L.ADG_SCEN_TWO_BUBBLES)
    dt = m.stable_dt(0.25)
    uo = o.step(u, dt)
    m.step(dt)
    a = m.get_state().cpu()
    if prec == L.ADG_PREC_FP64:
        # the finest leaves (level 2) set the floor's cell size
        fine = atmosphere_config(degree=5, nx=27 * 9, ny=27 * 9)
        _close(a, uo, floor=momentum_floor(fine, dt, 1, a[:, 0].numel()))
    else:
        assert _theta_err(o, a, uo) <= THETA_TOL
        assert (torch.linalg.vector_norm(a[:, 0] - uo[:, 0]) / torch.linalg.vector_norm(uo[:, 0])).item() <= 1e-9
