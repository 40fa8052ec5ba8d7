"""Pins of the oracle's local time stepping across the levels of the 3:1 tree
(oracle/amr.py step_lts, reading L1; not in the paper): the sub-interval
time weights, reduction to the global step on one level, conservation of
every integral across hanging faces and sub-steps, free-stream preservation,
accuracy against an exact Euler solution at the level of the global-step
run, and planted slips (wrong flux weight, full-step coarse traces) that
the pins catch."""
import math

import numpy as np
import pytest
import torch

from oracle.amr import AmrSolver
from oracle import physics as ph
from paper_1905_05524_gb300 import inputs


def wave(x, y, t, P, amp=0.2, U=1.0, L=6.0):
    """Exact Euler solution: a density wave advected at u = v = U, p = 1."""
    rho = 1.0 + amp * torch.sin(2 * math.pi * (x + y - 2 * U * t) / L)
    u = U + 0 * rho
    return [rho, rho * u, rho * u, 1.0 / (P.gamma - 1) + rho * u * u]


def _tree(N=2, mu=0.05, nx=6, seed=1, frac=0.3, levels=1):
    P = ph.cfd_params(N, mu=mu, source="none")
    a = AmrSolver(nx, nx, P, 6.0, 6.0, bc="periodic", max_level=levels)
    u = a.interpolate_field(lambda X, Y: wave(X, Y, 0.0, P))
    for lv in range(levels):
        flags = (torch.from_numpy(inputs.uniform_values(len(a.leaves), seed=seed + lv, lo=0, hi=1)) < frac).int()
        u = a.adapt(u, flags)
    return a, u


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_time_thirds_weights(N):
    """The three thirds' averages of the nodal time interpolant: their mean is
    the full-step average (weights w), and each is exact on t^m, m <= N."""
    a = AmrSolver(2, 2, ph.cfd_params(N, source="none"), 2.0, 2.0, bc="periodic")
    W = a.time_thirds()
    assert torch.allclose(W.sum(0) / 3.0, a.b.w, atol=1e-15)
    xi = a.b.xi
    for m in range(N + 1):
        for s in range(3):
            exact = 3.0 * (((s + 1) / 3.0) ** (m + 1) - (s / 3.0) ** (m + 1)) / (m + 1)
            assert abs(float((W[s] * xi ** m).sum()) - exact) <= 1e-14


def test_single_level_equals_global_step():
    P = ph.cfd_params(3, mu=0.05, source="none")
    a = AmrSolver(5, 4, P, 6.0, 6.0, bc="periodic")
    u = a.interpolate_field(lambda X, Y: wave(X, Y, 0.0, P))
    u = u + torch.from_numpy(inputs.perturbation(tuple(u.shape), seed=3, scale=0.01))
    ul, T = a.step_lts(u, 0.01)
    assert T == 0.01
    assert (ul - a.step(u, 0.01)).abs().max().item() <= 1e-14 * u.abs().max().item()


@pytest.mark.parametrize("levels", [1, 2])
def test_conservation_across_levels(levels):
    """Periodic trees with two and three levels: every integral is conserved
    to rounding over local-time-stepping cycles."""
    a, u = _tree(N=2, levels=levels, frac=0.35)
    assert len(a.levels()) == levels + 1
    u = u + torch.from_numpy(inputs.perturbation(tuple(u.shape), seed=5, scale=0.01))
    I0 = a.integral(u)
    for _ in range(2):
        u, _ = a.step_lts(u, 0.002 / 3 ** (levels - 1))   # stable on the finest level (viscous limit)
    I1 = a.integral(u)
    assert ((I1 - I0).abs() <= 2e-14 * I0.abs().clamp(min=1.0)).all(), (I1 - I0)


def test_free_stream_preserved():
    a, u = _tree(N=3, levels=2, frac=0.3)
    c = torch.zeros_like(u)
    c[:, 0], c[:, 1], c[:, 2], c[:, 3] = 1.2, 0.3, -0.2, 2.5
    v, _ = a.step_lts(c, 0.0005)   # stable on the finest level (viscous limit ~7e-4)
    assert (v - c).abs().max().item() <= 1e-13


def _error_at(a, u, dt, T, lts):
    P = a.P
    t = 0.0
    while t < T - 1e-12:
        if lts:
            u, dT = a.step_lts(u, dt, t)
        else:
            u, dT = a.step(u, dt, t), dt
        t += dT
    X, Y = a.node_coords()
    ex = torch.stack(wave(X, Y, t, P), 1)
    return (u - ex)[:, 0].abs().max().item(), t


def test_accuracy_matches_global_step():
    """Inviscid density wave on a two-level periodic tree, degree 3, to
    t = 0.189 (7 cycles, 21 steps of the finest level): the local-time-stepping
    error against the exact solution is within 1.5x of the global-step
    error on the same tree (coarse cells take 3x longer steps)."""
    a, u0 = _tree(N=3, mu=0.0, levels=1, frac=0.35)
    dt = 0.009
    e_lts, t1 = _error_at(a, u0.clone(), dt, 0.189, True)
    e_glb, t2 = _error_at(a, u0.clone(), dt, 0.189, False)
    assert abs(t1 - t2) < 1e-12
    assert e_lts <= 1.5 * e_glb, (e_lts, e_glb)
    assert e_lts < 1e-3


def test_planted_slips_fail(monkeypatch):
    """A wrong time weight on the accumulated fine fluxes breaks
    conservation; coarse traces over the whole coarse step instead of the
    sub-step's third degrade the accuracy pin."""
    import oracle.amr as am
    a, u = _tree(N=2, levels=1, frac=0.35)
    u = u + torch.from_numpy(inputs.perturbation(tuple(u.shape), seed=5, scale=0.01))
    I0 = a.integral(u)
    orig = am.AmrSolver._restrict_face
    monkeypatch.setattr(am.AmrSolver, "_restrict_face", lambda self, subs: orig(self, [s * 1.5 for s in subs]))
    v, _ = a.step_lts(u, 0.002)
    assert ((a.integral(v) - I0).abs() > 1e-10).any()
    monkeypatch.setattr(am.AmrSolver, "_restrict_face", orig)
    # full-step coarse traces for the fine side
    orig_tt = am.AmrSolver.time_thirds
    monkeypatch.setattr(am.AmrSolver, "time_thirds", lambda self: self.b.w[None, :].expand(3, -1).clone())
    b_, u0 = _tree(N=3, mu=0.0, levels=1, frac=0.35)
    e_bad, _ = _error_at(b_, u0.clone(), 0.009, 0.189, True)
    monkeypatch.setattr(am.AmrSolver, "time_thirds", orig_tt)
    e_good, _ = _error_at(b_, u0.clone(), 0.009, 0.189, True)
    assert e_bad > 1.5 * e_good, (e_bad, e_good)
