"""Linear stability of the oracle's step at the slip walls of Sec. 4.2
(reading C1).  The step is linearised at the resting isentropic atmosphere by
forward-mode differentiation of ``Solver.step`` on a 1x3 column of degree-5
cells (37 m, periodic in x, walls in y); its spectral radius decides
stability.  With the wall ghost that carries the background density and
energy (Eq. 10 reading R8) the step is stable up to CFL 0.46 of the dt rule
R11 and unstable at 0.5 with the growth factor the bubble runs show at the
bottom wall (~1.2 per step); a mirror ghost (interior density and energy) is
stable at 0.5, and so is the same column without gravity and walls.  So the
instability belongs to the ghost of Sec. 4.2 combined with the ADER step at
degree 5, and the warm-bubble workload runs at CFL 0.45."""
import numpy as np
import torch

from oracle.aderdg import Mesh, Solver
from oracle import physics as ph
from tests.oracle_bridge import background_field

H = 37.037


def _mirror_ghost(s):
    def ghost(tr, nrm, z):
        nx, ny = nrm
        rho, mx, my, E = tr["q"].unbind(1)
        mn = mx * nx + my * ny
        gq = [rho, mx - 2 * mn * nx, my - 2 * mn * ny, E]
        zero = torch.zeros_like(rho)
        F, G, _ = ph.fluxes(gq, tr["qx"].unbind(1), tr["qy"].unbind(1), z, s.P,
                            heat_override=(zero, zero + ph.dTbar_dz(s.P)))
        return torch.stack(gq, 1), torch.stack(F if nx != 0.0 else G, 1)
    return ghost


def spectral_radius(cfl, ghost="background", gravity=True):
    P = ph.atmosphere_params(5, mu=0.01)
    P.gravity = gravity
    bc_y = "wall" if gravity else "periodic"
    s = Solver(Mesh(1, 3, Lx=H, Ly=3 * H, bc_x="periodic", bc_y=bc_y), P)
    if ghost == "mirror":
        s._ghost = _mirror_ghost(s)
    if gravity:
        u0 = background_field(s)
    else:  # uniform air at rest, the sound speed of the atmosphere
        u0 = torch.zeros(3, 4, 6, 6, dtype=torch.float64)
        u0[:, 0] = 1.16
        u0[:, 3] = 1e5 / 0.4
    dt = s.stable_dt(u0, cfl)
    scale = torch.tensor([1.0, 1.0, 1.0, 1e3], dtype=torch.float64)[None, :, None, None].expand_as(u0)
    J = torch.func.jacfwd(lambda x: s.step(u0 + x * scale, dt) / scale)(torch.zeros_like(u0))
    J = J.reshape(u0.numel(), u0.numel()).numpy()
    return float(np.abs(np.linalg.eigvals(J)).max())


def test_background_ghost_stable_at_045_unstable_at_05():
    assert spectral_radius(0.45) <= 1.0 + 1e-7
    assert spectral_radius(0.46) <= 1.0 + 1e-7
    assert spectral_radius(0.5) >= 1.15


def test_mirror_ghost_and_interior_stable_at_05():
    assert spectral_radius(0.5, ghost="mirror") <= 1.0 + 1e-4
    assert spectral_radius(0.5, gravity=False) <= 1.0 + 1e-4


def test_background_ghost_semidiscrete_dissipative():
    """For linear acoustics (unit density and sound speed, state (p, u)) the
    Rusanov flux against the background ghost (p = 0, u reflected) puts
    -p^2/2 + p u/2 - u^2 into the boundary term of the energy balance: a
    negative definite form, so the semi-discrete scheme is dissipative and
    the instability above is one of the fully discrete step."""
    Q = np.array([[-0.5, 0.25], [0.25, -1.0]])
    assert np.linalg.eigvalsh(Q).max() < 0.0
