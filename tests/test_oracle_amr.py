"""Pins of the oracle's adaptive 3:1 tree (oracle/amr.py): transfer
operators, conservation across hanging faces and adaptation, equivalence of
a fully refined tree with the uniform fine mesh, 2-level balance."""
import math

import pytest
import torch

from oracle.amr import AmrSolver
from oracle.aderdg import Mesh, Solver
from oracle import physics as ph
from paper_1905_05524_gb300 import inputs


def density_wave(x, y, P, amp=0.2, U=1.0, L=6.0):
    rho = 1.0 + amp * torch.sin(2 * math.pi * (x + y) / L)
    u = U + 0 * rho
    return [rho, rho * u, rho * u, 1.0 / (P.gamma - 1) + rho * u * u]


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_restrict_prolong_identity_and_polynomial_exactness(N):
    a = AmrSolver(3, 3, ph.cfd_params(N, source="none"), 3.0, 3.0, bc="periodic")
    n = N + 1
    u = torch.from_numpy(inputs.perturbation((4, n, n), seed=N, scale=1.0))
    kids = a.prolong_cell(u)
    assert torch.allclose(a.restrict_cell(kids), u, atol=1e-13)
    # prolongation of a degree-N polynomial = the polynomial at the children's nodes
    xi = a.b.xi
    f = lambda x, y: (1 + 2 * x - x ** N) * (0.5 - y + 3 * y ** N)
    par = f(xi[None, :], xi[:, None])[None].expand(4, n, n)
    for (ca, cb), uc in a.prolong_cell(par).items():
        ref = f((ca + xi[None, :]) / 3, (cb + xi[:, None]) / 3)
        assert torch.allclose(uc[0], ref, atol=1e-12)


def _random_refined(a, seed, frac=0.3):
    flags = (torch.from_numpy(inputs.uniform_values(len(a.leaves), seed=seed, lo=0, hi=1)) < frac).int()
    return flags


def test_conservation_with_hanging_faces():
    """Periodic tree with refined patches: every integral is conserved to
    rounding over steps (hanging faces included) and across adaptation."""
    P = ph.cfd_params(2, mu=0.05, source="none")
    a = AmrSolver(6, 6, P, 6.0, 6.0, bc="periodic", max_level=2)
    u = a.interpolate_field(lambda X, Y: density_wave(X, Y, P))
    u = a.adapt(u, _random_refined(a, 1))
    u = a.adapt(u, _random_refined(a, 2, 0.15))
    assert len({c[0] for c in a.leaves}) >= 2
    I0 = a.integral(u)
    for _ in range(3):
        u = a.step(u, 0.004)
    I1 = a.integral(u)
    assert ((I1 - I0).abs() <= 1e-13 * I0.abs().clamp(min=1.0)).all(), (I1 - I0)
    # coarsen everything that can be coarsened: integrals unchanged
    u2 = a.adapt(u, torch.full((len(a.leaves),), -1))
    assert ((a.integral(u2) - I1).abs() <= 1e-13 * I1.abs().clamp(min=1.0)).all()


def test_fully_refined_tree_equals_uniform_fine_mesh():
    P = ph.cfd_params(2, mu=0.05, source="none")
    a = AmrSolver(3, 3, P, 6.0, 6.0, bc="periodic", max_level=1)
    u = a.interpolate_field(lambda X, Y: density_wave(X, Y, P))
    u = a.adapt(u, torch.ones(9, dtype=torch.int64))
    assert all(c[0] == 1 for c in a.leaves) and len(a.leaves) == 81
    s = Solver(Mesh(9, 9, Lx=6.0, Ly=6.0), P)
    uf = s.interpolate(lambda x, y, t, P_: density_wave(x, y, P_))
    # the leaves are in row-major order of the fine mesh: start both from uf
    X, Y = a.node_coords()
    assert torch.allclose(X, s.X, atol=1e-14) and torch.allclose(Y, s.Y, atol=1e-14)
    u = uf.clone()
    for _ in range(2):
        u = a.step(u, 0.005)
        uf = s.step(uf, 0.005)
    assert torch.allclose(u, uf, rtol=1e-12, atol=1e-13)


def test_balance_rule():
    """Refining one cell twice forces its neighbours to keep every face at a
    level difference of at most one."""
    P = ph.cfd_params(2, source="none")
    a = AmrSolver(5, 5, P, 5.0, 5.0, bc="wall", max_level=2)
    u = a.interpolate_field(lambda X, Y: density_wave(X, Y, P))
    fl = torch.zeros(25, dtype=torch.int64)
    fl[12] = 1
    u = a.adapt(u, fl)
    fl = torch.tensor([1 if c == (1, 7, 7) else 0 for c in a.leaves])
    u = a.adapt(u, fl)
    for k, c in enumerate(a.leaves):
        for f in "EWNS":
            nb = a.neighbour(c, f)   # raises for an unbalanced tree
            if nb[0] == "conf":
                assert a.leaves[nb[1]][0] == c[0]
    assert max(c[0] for c in a.leaves) == 2


def test_hydrostatic_balance_with_hanging_faces():
    """The background atmosphere on a tree with hanging faces and slip walls
    stays at rest to 1e-9 over 20 steps."""
    P = ph.atmosphere_params(3)
    a = AmrSolver(6, 6, P, 1000.0, 1000.0, bc="wall", max_level=1)
    X, Y = a.node_coords()
    u = torch.stack(ph.bubble_state(X, Y, 0 * X, P), 1)
    fl = torch.zeros(36, dtype=torch.int64)
    fl[[7, 8, 14, 21]] = 1
    u = a.adapt(u, fl)
    X, Y = a.node_coords()
    u = torch.stack(ph.bubble_state(X, Y, 0 * X, P), 1)
    for _ in range(20):
        u = a.step(u, 0.002)
    vel = (u[:, 1:3] / u[:, 0:1]).abs().max().item()
    assert vel < 1e-9, vel
