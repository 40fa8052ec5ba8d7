"""Mixed-precision MUSCL-Hancock finite volumes (adg_fv_* with ADG_PREC_MIXED):
FP64 state, FP32 arithmetic on perturbations of the hydrostatic background,
FP64 accumulation, one fused tile kernel per step; against the FP64 oracle
(oracle/fv.py, readings FV1-FV5).

Bounds.  Every FP32 operation rounds with relative error u = 2^-24; one step
is a chain of O(10) operations on perturbation-sized values, so a step adds
an error of about 10 u relative to the perturbation, and K steps at most
K * 10 u (errors of one sign), typically sqrt(K) * 10 u.  With K <= 20:
relative L2 of theta' and of rho' <= 20 * 10 * 2^-24 ~ 1.2e-5; taken as
THETA_TOL = 1.5e-5, also for momentum, floored at 1 m/s * |rho| (the
bubbles start at rest, and p' = (gamma - 1)(E' - ke - g z rho') cancels
E' ~ g z rho' in FP32, an absolute error that does not shrink with the flow
speed).  The FP64 parts (total rho) stay within 1e-9 relative.
Without gravity the FP32 path carries the whole state: relative L2 per
variable <= FULL_TOL = 1e-5 after 10 steps."""
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300.solver import FvMesh, MeshConfig, fv_bubble_config
from oracle import physics as ph
from tests.test_gpu_fv import oracle, bubbles, random_state

pytestmark = pytest.mark.gpu

THETA_TOL = 1.5e-5
FULL_TOL = 1e-5


def mixed(cfg):
    cfg.precision = L.ADG_PREC_MIXED
    return cfg


def theta_prime(o, U):
    return ph.theta(list(U.unbind(0)), o.zc, o.P) - o.P.theta0


def rel(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


def check_bubble(o, a, b, tol=THETA_TOL):
    a = a.detach().cpu().double()
    rb = o.background_state(o.zc)[0]
    et = rel(theta_prime(o, a), theta_prime(o, b))
    er = rel(a[0] - rb, b[0] - rb)
    nrho = torch.linalg.vector_norm(b[0]).item()
    em = max(torch.linalg.vector_norm(a[v] - b[v]).item() / max(torch.linalg.vector_norm(b[v]).item(), nrho)
             for v in (1, 2))
    assert et <= tol, f"theta' rel L2 {et:.3e}"
    assert er <= tol, f"rho' rel L2 {er:.3e}"
    assert em <= tol, f"momentum rel L2 {em:.3e}"
    assert rel(a[0], b[0]) <= 1e-9
    return et, er, em


def stirred_bubbles(o, seed):
    """The two bubbles (Eq. 14) plus seeded cell-level noise: velocity up to
    1 m/s and rho' up to 1e-4 kg/m^3 (rhoE adjusted to keep p), so every
    flux, limiter branch and wall ghost is active from the first step."""
    from paper_1905_05524_gb300 import inputs
    U = bubbles(o)
    n = inputs.perturbation((3, o.ny, o.nx), seed, 1.0)
    noise = torch.from_numpy(n)
    rho = U[0] + 1e-4 * noise[2]
    p = ph.pressure(list(U.unbind(0)), o.zc, o.P)
    u, v = noise[0], noise[1]
    E = p / (o.P.gamma - 1.0) + 0.5 * rho * (u * u + v * v) + rho * o.P.g * o.zc
    return torch.stack([rho, rho * u, rho * v, E], 0)


@pytest.mark.parametrize("nx,ny", [(41, 37), (32, 8), (70, 20), (1, 5), (3, 2)])
def test_mixed_two_bubbles_walls_match_oracle(nx, ny):
    """Ragged and exact tiles (32 x 8 cells per tile), walls on all sides,
    20 steps at CFL 0.5 from the stirred bubbles."""
    cfg = mixed(fv_bubble_config(nx=nx, ny=ny))
    o = oracle(cfg)
    U = stirred_bubbles(o, nx * 31 + ny)
    dt = o.stable_dt(U, 0.5)
    m = FvMesh(cfg)
    m.set_state(U)
    assert abs(m.stable_dt(0.5) - dt) <= 1e-13 * dt
    for _ in range(20):
        U = o.step(U, dt)
    m.step(dt, 20)
    check_bubble(o, m.get_state(), U)


def test_mixed_full_size_bubbles_match_oracle():
    """The timed configuration: 630 x 630 cells (7^2 patches of 90^2), the
    colliding bubbles from the device initialisation, 3 steps at CFL 0.5,
    every cell compared."""
    cfg = mixed(fv_bubble_config(nx=630, ny=630))
    o = oracle(cfg)
    m = FvMesh(cfg)
    m.init_scenario(L.ADG_SCEN_TWO_BUBBLES)
    U = m.get_state().cpu()
    assert rel(U, bubbles(o)) <= 1e-14
    dt = m.stable_dt(0.5)
    m.step(dt, 3)
    for _ in range(3):
        U = o.step(U, dt)
    check_bubble(o, m.get_state(), U)


def test_mixed_steps_resume_after_odd_counts_and_set_state():
    """The fused step writes the second state buffer and swaps: state reads
    and writes between odd and even step counts see the current state."""
    cfg = mixed(fv_bubble_config(nx=45, ny=19))
    o = oracle(cfg)
    U0 = stirred_bubbles(o, 5)
    dt = o.stable_dt(U0, 0.5)
    m = FvMesh(cfg)
    m.set_state(U0)
    m.step(dt, 1)
    U1 = o.step(U0, dt)
    check_bubble(o, m.get_state(), U1)
    m.step(dt, 2)
    U3 = o.step(o.step(U1, dt), dt)
    check_bubble(o, m.get_state(), U3)
    m.set_state(U0)
    m.step(dt, 1)
    check_bubble(o, m.get_state(), U1)


def test_mixed_atmosphere_at_rest_and_bitwise_repeatable():
    cfg = mixed(fv_bubble_config(nx=40, ny=24))
    outs = []
    for _ in range(2):
        m = FvMesh(cfg)
        m.init_scenario(L.ADG_SCEN_BACKGROUND)
        dt = m.stable_dt(0.5)
        m.step(dt, 20)
        outs.append(m.get_state().cpu())
    a = outs[0]
    assert torch.equal(outs[0], outs[1])
    assert (a[1:3] / a[0]).abs().max().item() <= 1e-9


@pytest.mark.parametrize("nx,ny", [(15, 11), (33, 9), (1, 1), (64, 3)])
def test_mixed_periodic_random_state_matches_oracle(nx, ny):
    """No gravity, periodic in x and y: the FP32 path carries the whole
    state.  Relative L2 per variable <= FULL_TOL after 10 steps; mass,
    momentum and energy integrals kept to 1e-6 relative (FP32 flux
    differences, FP64 sums)."""
    cfg = mixed(MeshConfig(degree=1, nx=nx, ny=ny, Lx=2.0, Ly=1.5, mu=0.0))
    o = oracle(cfg)
    U = random_state(o, nx * 7 + ny)
    I0 = o.integral(U)
    dt = o.stable_dt(U, 0.5)
    m = FvMesh(cfg)
    m.set_state(U)
    for _ in range(10):
        U = o.step(U, dt)
    m.step(dt, 10)
    a = m.get_state().cpu()
    for v in range(4):
        r = torch.linalg.vector_norm(a[v] - U[v]).item() / max(torch.linalg.vector_norm(U[v]).item(), 1e-300)
        assert r <= FULL_TOL, (v, r)
    Ia = o.integral(a)
    assert ((Ia - I0).abs() <= 1e-6 * I0.abs().clamp(min=1.0)).all(), (Ia - I0)


def test_mixed_rejects_gravity_with_periodic_y():
    cfg = mixed(fv_bubble_config(nx=8, ny=8))
    cfg.bc_y = L.ADG_BC_PERIODIC
    with pytest.raises(L.AdgError):
        FvMesh(cfg)
