"""Pins of the oracle's point-wise physics (Sec. 2) against textbook forms,
independent autograd derivatives and the paper's printed constants."""
import json
import math
import os

import torch

from oracle import physics as ph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
T64 = dict(dtype=torch.float64)


def test_paper_constants_golden():
    g = json.load(open(GOLDEN))
    P = ph.cfd_params(3)
    assert P.gamma == g["cfd_constants"]["gamma"] and P.Pr == g["cfd_constants"]["Pr"]
    assert abs(P.cv - g["cfd_constants"]["c_v"]) < 1e-15
    A = ph.atmosphere_params(5)
    for k in ("gamma", "Pr", "R", "p0"):
        assert getattr(A, k) == g["atmosphere"][k]
    # two-bubble and cosine parameters as printed (Eqs. 14, 16)
    x = torch.tensor([500.0, 560.0], **T64)
    z = torch.tensor([300.0, 640.0], **T64)
    tb = ph.two_bubbles(x, z)
    w, c = g["two_bubbles"]["warm"], g["two_bubbles"]["cold"]
    # at the warm centre the cold bubble contributes A_c exp(-r^2/s^2)
    r = math.hypot(w["xc"] - c["xc"], w["zc"] - c["zc"])
    assert abs(tb[0].item() - (w["A"] + c["A"] * math.exp(-(r - c["a"]) ** 2 / c["s"] ** 2))) < 1e-15
    cb = g["cosine_bubble"]
    val = ph.cosine_bubble(torch.tensor([cb["xc"]], **T64), torch.tensor([cb["zc"]], **T64))
    assert abs(val.item() - cb["A"]) < 1e-15
    edge = ph.cosine_bubble(torch.tensor([cb["xc"] + cb["a"]], **T64), torch.tensor([cb["zc"]], **T64))
    assert abs(edge.item()) < 1e-15
    d = g["scalability_dof"]
    dof = d["cells_per_side"] ** 2 * d["nodes_per_side"] ** 2 * d["vars"]
    assert abs(dof - d["approx_dof"]) / d["approx_dof"] < 0.01


def test_background_is_hydrostatic():
    """Eq. 6: d pbar/dz = -g rhobar (central difference, h = 1e-3 m)."""
    P = ph.atmosphere_params(3)
    z = torch.linspace(0.0, 1000.0, 11, **T64)
    h = 1e-3
    pp, _, _ = ph.background(z + h, P)
    pm, _, _ = ph.background(z - h, P)
    _, rho, T = ph.background(z, P)
    dp = (pp - pm) / (2 * h)
    assert torch.allclose(dp, -P.g * rho, rtol=1e-8)
    # potential temperature of the background is theta0 (constant)
    pb, rb, Tb = ph.background(z, P)
    E = pb / (P.gamma - 1.0) + rb * P.g * z
    q = [rb, 0 * rb, 0 * rb, E]
    assert torch.allclose(ph.theta(q, z, P), torch.full_like(z, P.theta0), rtol=1e-13)


def test_bubble_state_theta_and_pressure():
    P = ph.atmosphere_params(5)
    x = torch.linspace(0, 1000, 7, **T64)
    z = torch.linspace(0, 1000, 7, **T64)
    th = ph.cosine_bubble(x, z, 0.5, 250.0, 500.0, 350.0)
    q = ph.bubble_state(x, z, th, P)
    assert torch.allclose(ph.theta(q, z, P), P.theta0 + th, rtol=0, atol=1e-11)
    pb, _, _ = ph.background(z, P)
    assert torch.allclose(ph.pressure(q, z, P), pb, rtol=1e-13)


def test_euler_flux_of_uniform_state():
    """Zero gradients, no gravity: the hyperbolic flux of Eq. 1 (Euler)."""
    P = ph.cfd_params(3, mu=0.3)
    rho, u, v, p = 1.3, 0.7, -0.2, 2.0
    E = p / (P.gamma - 1) + 0.5 * rho * (u * u + v * v)
    q = [torch.tensor(a, **T64) for a in (rho, rho * u, rho * v, E)]
    z0 = [torch.tensor(0.0, **T64)] * 4
    F, G, S = ph.fluxes(q, z0, z0, torch.tensor(0.0, **T64), P)
    ref_F = [rho * u, rho * u * u + p, rho * u * v, u * (E + p)]
    ref_G = [rho * v, rho * u * v, rho * v * v + p, v * (E + p)]
    for a, b in zip(F + G, ref_F + ref_G):
        assert abs(a.item() - b) < 1e-14
    assert all(abs(s.item()) == 0 for s in S)


def _primitive_fluxes(x, y, P):
    """Viscous NS flux from primitive fields differentiated directly by
    autograd (no chain rule through conserved gradients)."""
    rho = 1.0 + 0.2 * torch.sin(x + 2 * y)
    u = 0.3 * torch.cos(2 * x - y)
    v = -0.1 + 0.2 * torch.sin(x * y)
    p = 1.0 + 0.1 * torch.cos(x) * torch.sin(y)
    grad = lambda f: torch.autograd.grad(f.sum(), [x, y], create_graph=True)
    ux, uy = grad(u)
    vx, vy = grad(v)
    T = p / (rho * P.R)
    Tx, Ty = grad(T)
    div = ux + vy
    sxx = P.mu * (2 / 3 * div - 2 * ux)
    syy = P.mu * (2 / 3 * div - 2 * vy)
    sxy = -P.mu * (uy + vx)
    E = p / (P.gamma - 1) + 0.5 * rho * (u * u + v * v)
    F = [rho * u, rho * u * u + p + sxx, rho * u * v + sxy, u * (E + p) + u * sxx + v * sxy - P.kappa * Tx]
    G = [rho * v, rho * u * v + sxy, rho * v * v + p + syy, v * (E + p) + u * sxy + v * syy - P.kappa * Ty]
    return [rho, rho * u, rho * v, E], F, G


def test_viscous_flux_chain_rule_matches_primitive_autograd():
    """Reading R5 (gradients of v, p, T from grad Q by the chain rule) against
    the stress tensor (Eq. 4) and heat flux (Eq. 5) of primitive fields."""
    P = ph.cfd_params(3, mu=0.37)
    x = torch.linspace(0.1, 2.0, 9, **T64).requires_grad_(True)
    y = torch.linspace(-1.0, 0.7, 9, **T64).requires_grad_(True)
    Q, Fr, Gr = _primitive_fluxes(x, y, P)
    Qx, Qy = [], []
    for c in Q:
        gx, gy = torch.autograd.grad(c.sum(), [x, y], retain_graph=True)
        Qx.append(gx)
        Qy.append(gy)
    F, G, _ = ph.fluxes(Q, Qx, Qy, y, P)
    for a, b in zip(F + G, Fr + Gr):
        assert torch.allclose(a, b, rtol=1e-12, atol=1e-13)


def test_steady_manufactured_source_closed_form():
    """Autograd source of the steady field equals the hand-derived form
    S = 2 U a k cos(k s) (1, U, U, U^2) - kappa Laplace(p/(rho R))."""
    P = ph.cfd_params(3, mu=0.1, source="steady")
    x = torch.linspace(0, 10, 13, **T64)
    y = torch.linspace(0, 10, 13, **T64).flip(0)
    S = ph.manufactured_source(x, y, 0.0, P)
    a, U, k, p = 0.1, 0.5, 2 * math.pi / 10, 1.0
    s = x + y
    rho = 1 + a * torch.sin(k * s)
    c = 2 * U * a * k * torch.cos(k * s)
    lapT = (2 * p / P.R) * (a * k * k * torch.sin(k * s) / rho ** 2 + 2 * a * a * k * k * torch.cos(k * s) ** 2 / rho ** 3)
    ref = [c, c * U, c * U, c * U * U - P.kappa * lapT]
    for a_, b_ in zip(S, ref):
        assert torch.allclose(a_, b_, rtol=1e-12, atol=1e-13)


def test_gravity_source_and_perturbation_split():
    """Eq. 7: momentum flux carries p' = p - pbar, source -g rho'."""
    P = ph.atmosphere_params(3)
    z = torch.tensor([123.0], **T64)
    pb, rb, _ = ph.background(z, P)
    rho = rb * 1.001
    E = pb * 1.0005 / (P.gamma - 1) + rho * P.g * z
    q = [rho, 0 * rho, 0 * rho, E]
    zero = [0 * rho] * 4
    F, G, S = ph.fluxes(q, zero, zero, z, P)
    p = ph.pressure(q, z, P)
    assert torch.allclose(G[2], p - pb, rtol=1e-12)
    assert torch.allclose(S[2], -P.g * (rho - rb), rtol=1e-12)
    assert torch.allclose(F[3] * 0, F[3])  # fluid at rest: zero energy flux
