"""GPU (libaderdg.so through the C ABI) vs the FP64 CPU oracle, element by
element on the same seeded inputs.

Tolerance (FP64 path): relative L2 per variable <= 1e-11 against the oracle.
The momentum components add the rounding floor of tests/tolerances.py: in a
fluid at rest over a hydrostatic background the momentum is driven by
p' = p - pbar, which both implementations form by cancelling O(1e5 Pa)
values, so their momenta differ by the FP64 rounding of that difference
carried through the face lifting, not by the size of the (near-zero)
momentum.  The bubble tests print the raw per-variable differences.
"""
import math

import numpy as np
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.solver import Mesh, MeshConfig, atmosphere_config, steady_manufactured_config
from tests.oracle_bridge import oracle_for, steady_field, cosine_field, two_bubble_field, background_field
from tests.tolerances import momentum_floor
from oracle import indicator as oind

pytestmark = pytest.mark.gpu

TOL = 1e-11


def rel_l2(a, b):
    """Per-variable relative L2 of a (GPU) against b (oracle), both [c, v, j, i]."""
    a = a.detach().cpu().double()
    b = b.detach().cpu().double()
    out = []
    for v in range(4):
        d = torch.linalg.vector_norm(a[:, v] - b[:, v]).item()
        nb = torch.linalg.vector_norm(b[:, v]).item()
        out.append(d / max(nb, 1e-300))
    return out


def assert_close(a, b, tol=TOL, what="", floor=0.0):
    """Per-variable L2: |a - b| <= tol |b|, plus `floor` (absolute, the
    rounding floor of tests/tolerances.py) for the momentum components."""
    a = a.detach().cpu().double()
    b = b.detach().cpu().double()
    for v in range(4):
        d = torch.linalg.vector_norm(a[:, v] - b[:, v]).item()
        nb = torch.linalg.vector_norm(b[:, v]).item()
        bound = tol * nb + (floor if v in (1, 2) else 0.0)
        if floor:
            print(f"{what} var {v}: |d| = {d:.3e}, |ref| = {nb:.3e}, relative {d / max(nb, 1e-300):.3e}, "
                  f"bound {bound:.3e}")
        assert d <= max(bound, 1e-300 * nb), \
            f"{what} var {v}: |d|={d:.3e} |ref|={nb:.3e} rel={d / max(nb, 1e-300):.3e} bound={bound:.3e}"


def floor_for(cfg, dt, steps):
    return momentum_floor(cfg, dt, steps, cfg.nx * cfg.ny * (cfg.degree + 1) ** 2)


def run_pair(cfg, u0, dt, steps):
    """Run GPU and oracle from the same initial state u0 (oracle tensor)."""
    m = Mesh(cfg)
    m.set_state(u0.to("cuda").contiguous())
    o = oracle_for(cfg)
    uo = u0.clone()
    t = 0.0
    for _ in range(steps):
        uo = o.step(uo, dt, t)
        t += dt
    m.step(dt, steps)
    torch.cuda.synchronize()
    return m.get_state().cpu(), uo, m, o


def test_init_steady_matches_oracle():
    cfg = steady_manufactured_config(degree=3, nx=9, ny=9)
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_STEADY)
    o = oracle_for(cfg)
    assert_close(m.get_state(), steady_field(o, cfg), 1e-14, "init steady")


def test_init_cosine_bubble_matches_oracle():
    cfg = atmosphere_config(degree=5, nx=9, ny=9)
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    o = oracle_for(cfg)
    assert_close(m.get_state(), cosine_field(o), 1e-13, "init cosine")


def test_init_two_bubbles_matches_oracle():
    cfg = atmosphere_config(degree=3, nx=27, ny=27)
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_TWO_BUBBLES)
    o = oracle_for(cfg)
    assert_close(m.get_state(), two_bubble_field(o), 1e-13, "init two bubbles")


@pytest.mark.parametrize("degree", [1, 2, 3, 4, 5, 6, 7])
def test_step_steady_manufactured_all_degrees(degree):
    """C1-type periodic manufactured run, every degree, 9x9 cells (ragged tail
    for every cells-per-block choice), 3 steps."""
    cfg = steady_manufactured_config(degree=degree, nx=9, ny=9)
    o = oracle_for(cfg)
    u0 = steady_field(o, cfg)
    u0 = u0 + torch.from_numpy(inputs.perturbation(tuple(u0.shape), seed=10 + degree, scale=1e-3))
    dt = o.stable_dt(u0, 0.5)
    a, b, _, _ = run_pair(cfg, u0, dt, 3)
    assert_close(a, b, what=f"N={degree}")


def test_step_steady_manufactured_9x9_20_steps():
    """Steady manufactured case: N = 3, 9x9 periodic [0,10]^2, steady manufactured, CFL 0.5, 20 steps."""
    cfg = steady_manufactured_config(degree=3, nx=9, ny=9)
    o = oracle_for(cfg)
    u0 = steady_field(o, cfg)
    dt = o.stable_dt(u0, 0.5)
    a, b, _, _ = run_pair(cfg, u0, dt, 20)
    assert_close(a, b, what="steady manufactured 9x9")


def test_stable_dt_matches_oracle():
    cfg = steady_manufactured_config(degree=3, nx=9, ny=9)
    o = oracle_for(cfg)
    u0 = steady_field(o, cfg)
    m = Mesh(cfg)
    m.set_state(u0.cuda().contiguous())
    assert abs(m.stable_dt(0.5) - o.stable_dt(u0, 0.5)) <= 1e-14 * o.stable_dt(u0, 0.5)


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 3), (3, 1)])
def test_tiny_periodic_grids(nx, ny):
    cfg = steady_manufactured_config(degree=2, nx=nx, ny=ny)
    cfg.Lx, cfg.Ly = 10.0 * nx / 3, 10.0 * ny / 3
    o = oracle_for(cfg)
    u0 = steady_field(o, cfg)
    u0 = u0 + torch.from_numpy(inputs.perturbation(tuple(u0.shape), seed=3, scale=1e-2))
    dt = o.stable_dt(u0, 0.5)
    a, b, _, _ = run_pair(cfg, u0, dt, 4)
    assert_close(a, b, what=f"{nx}x{ny}")


def test_bubble_walls_small():
    """Atmosphere with slip walls, cosine bubble, N = 5 on 9x9, 5 steps."""
    cfg = atmosphere_config(degree=5, nx=9, ny=9)
    o = oracle_for(cfg)
    u0 = cosine_field(o)
    dt = o.stable_dt(u0, 0.5)
    a, b, _, _ = run_pair(cfg, u0, dt, 5)
    assert_close(a, b, what="bubble 9x9", floor=floor_for(cfg, dt, 5))


def test_bubble_momentum_floor_catches_planted_error():
    """A momentum error of ten times the rounding floor, planted in the
    oracle's result, fails the bubble comparison; the floor is 50x tighter
    than 1e-11 x |rho| x 1 m/s here."""
    cfg = atmosphere_config(degree=5, nx=9, ny=9)
    o = oracle_for(cfg)
    u0 = cosine_field(o)
    dt = o.stable_dt(u0, 0.5)
    a, b, _, _ = run_pair(cfg, u0, dt, 5)
    fl = floor_for(cfg, dt, 5)
    nodes = b[:, 1].numel()
    for v in (1, 2):
        bad = b.clone()
        bad[:, v] += 10.0 * fl / nodes ** 0.5
        with pytest.raises(AssertionError):
            assert_close(a, bad, what="planted", floor=fl)
    assert fl <= 0.05 * 1e-11 * torch.linalg.vector_norm(b[:, 0]).item()


def test_two_bubbles_walls_degree3():
    cfg = atmosphere_config(degree=3, nx=27, ny=27, mu=0.001)
    o = oracle_for(cfg)
    u0 = two_bubble_field(o)
    dt = o.stable_dt(u0, 0.5)
    a, b, _, _ = run_pair(cfg, u0, dt, 3)
    assert_close(a, b, what="two bubbles", floor=floor_for(cfg, dt, 3))


def test_warm_bubble_81x81_full_size_two_steps():
    """The warm bubble at full size (N = 5, 81x81, walls, cosine bubble), the launch
    configuration bench.py times: 2 steps compared element by element."""
    cfg = atmosphere_config(degree=5, nx=81, ny=81)
    o = oracle_for(cfg)
    u0 = cosine_field(o)
    dt = o.stable_dt(u0, 0.5)
    a, b, _, _ = run_pair(cfg, u0, dt, 2)
    assert_close(a, b, what="warm bubble 81x81", floor=floor_for(cfg, dt, 2))


def test_predictor_corrector_split_equals_step():
    cfg = steady_manufactured_config(degree=4, nx=5, ny=4)
    o = oracle_for(cfg)
    u0 = steady_field(o, cfg)
    m1, m2 = Mesh(cfg), Mesh(cfg)
    m1.set_state(u0.cuda().contiguous())
    m2.set_state(u0.cuda().contiguous())
    m1.step(0.01)
    m2.predictor(0.01)
    m2.corrector(0.01)
    assert torch.equal(m1.get_state(), m2.get_state())


def test_corrector_without_predictor_is_state_error():
    m = Mesh(steady_manufactured_config(degree=2, nx=3, ny=3))
    with pytest.raises(L.AdgError) as e:
        m.corrector(0.01)
    assert e.value.code == L.ADG_ESTATE
    m.predictor(0.01)
    with pytest.raises(L.AdgError):
        m.corrector(0.02)


def test_mass_conservation_and_determinism():
    """Periodic FP64: sum of quadrature-weighted mass is conserved to rounding;
    repeated runs are bitwise identical; 10 + 10 steps == 20 steps."""
    cfg = steady_manufactured_config(degree=3, nx=12, ny=10)
    o = oracle_for(cfg)
    u0 = steady_field(o, cfg) + torch.from_numpy(inputs.perturbation((120, 4, 4, 4), seed=5, scale=1e-2))
    dt = o.stable_dt(u0, 0.5)
    m = Mesh(cfg)
    m.set_state(u0.cuda().contiguous())
    m.step(dt, 20)
    a = m.get_state().cpu()
    I0, I1 = o.integral(u0), o.integral(a)
    assert abs(I1[0] - I0[0]) <= 1e-13 * abs(I0[0])
    m.set_state(u0.cuda().contiguous())
    m.step(dt, 10)
    mid = m.get_state()
    m2 = Mesh(cfg)
    m2.set_state(mid)
    m2.step(dt, 10)
    assert torch.equal(m2.get_state().cpu(), a)


def test_constant_state_preserved():
    cfg = MeshConfig(degree=4, nx=7, ny=6, source=L.ADG_SRC_NONE)
    c = torch.zeros((42, 4, 5, 5), dtype=torch.float64)
    c[:, 0], c[:, 1], c[:, 2], c[:, 3] = 1.3, 0.2, -0.4, 3.0
    m = Mesh(cfg)
    m.set_state(c.cuda())
    m.step(0.005, 10)
    assert (m.get_state().cpu() - c).abs().max().item() < 1e-13


def test_hydrostatic_background_gpu_matches_oracle():
    cfg = atmosphere_config(degree=3, nx=9, ny=9)
    o = oracle_for(cfg)
    u0 = background_field(o)
    dt = o.stable_dt(u0, 0.5)
    a, b, _, _ = run_pair(cfg, u0, dt, 10)
    # momenta are rounding noise here: compare absolutely against the momentum scale rho*1e-9
    for v in (0, 3):
        assert torch.linalg.vector_norm(a[:, v] - b[:, v]) <= TOL * torch.linalg.vector_norm(b[:, v])
    assert (a[:, 1:3] - b[:, 1:3]).abs().max().item() < 1e-9


@pytest.mark.parametrize("var,cfgname", [("theta", "bubble"), ("rho", "steady"), ("theta", "bubble_large"),
                                         ("rho", "steady_n1")])
def test_tv_indicator_matches_oracle(var, cfgname):
    # bubble_large: 1599 cells in 400 blocks of 4, so the statistics fold two
    # block triples per thread and the last block holds 3 cells; steady_n1:
    # blocks of 32 cells, the last holding 15
    if cfgname in ("bubble", "bubble_large"):
        cfg = atmosphere_config(degree=5, nx=27, ny=27) if cfgname == "bubble" else \
            atmosphere_config(degree=5, nx=41, ny=39)
        o = oracle_for(cfg)
        u0 = two_bubble_field(o)
    else:
        cfg = steady_manufactured_config(degree=3, nx=9, ny=9) if cfgname == "steady" else \
            steady_manufactured_config(degree=1, nx=13, ny=11)
        o = oracle_for(cfg)
        u0 = steady_field(o, cfg)
    m = Mesh(cfg)
    m.set_state(u0.cuda().contiguous())
    T_r, T_c = 2.5, -0.5
    tv, flags, (mean, std) = m.tv_indicator(L.ADG_TV_THETA if var == "theta" else L.ADG_TV_RHO, T_r, T_c)
    tvo, flo, meano, stdo = oind.tv_indicator(o, u0, var, T_r, T_c)
    tv = tv.cpu()
    # cells at rest carry TV ~1e-11 that is pure FP64 rounding of theta ~ 300 K
    # (eps * theta0 through the derivative): relative 1e-11 plus that floor
    floor = 1e-10 * tvo.abs().max()
    assert bool(((tv - tvo).abs() <= 1e-11 * tvo.abs() + floor).all()), (tv - tvo).abs().max()
    assert abs(mean - meano) <= 1e-11 * abs(meano) + floor
    assert abs(std - stdo) <= 1e-10 * abs(stdo) + floor
    # flags: identical except where TV sits within rounding of a threshold
    thr_r, thr_c = meano + T_r * stdo, meano + T_c * stdo
    amb = ((tvo - thr_r).abs() <= 1e-9 * abs(thr_r)) | ((tvo - thr_c).abs() <= 1e-9 * abs(thr_c))
    fl = flags.cpu()
    assert torch.equal(fl[~amb], flo[~amb])
    assert bool(((fl[amb] >= -1) & (fl[amb] <= 1)).all())


def test_check_finite():
    cfg = steady_manufactured_config(degree=2, nx=3, ny=3)
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_STEADY)
    m.check_finite()
    u = m.get_state()
    u[4, 1, 0, 0] = float("nan")
    m.set_state(u)
    with pytest.raises(L.AdgError) as e:
        m.check_finite()
    assert e.value.code == L.ADG_ENONFINITE


def test_state_ptr_view_aliases_state():
    cfg = steady_manufactured_config(degree=2, nx=3, ny=3)
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_STEADY)
    view = m.state_view()
    assert torch.equal(view, m.get_state())
    m.step(0.01)
    assert torch.equal(view, m.get_state())
