"""Point-wise physics of the 3D compressible Navier-Stokes system (oracle).

Sec. 2 of the paper in three dimensions, with the same readings as the 2D
module (physics.py): Q = (rho, rho u, rho v, rho w, rho E), gravity along the
third coordinate z;

* Eq. 2  p = (gamma-1)(rhoE - 1/2 |rho v|^2/rho - rho g z);
* Eq. 4  sigma = mu((2/3) div v I - (grad v + grad v^T));
* Eq. 5  kappa = mu c_p / Pr, heat flux -kappa grad T with p = rho R T;
* Eq. 7  momentum fluxes carry p' = p - pbar(z); the z-momentum source is
         -g rho' with rho' = rho - rhobar(z);
* Sec. 4.1 the ABC flow (an exact solution of the incompressible equations,
         imposed as initial and boundary data);
* Sec. 4.2 the 3D cosine bubble (yc = xc) on the isentropic background.

The flux in direction b is written once for all three directions:
    mass      rho v_b
    momentum  rho v_a v_b + delta_ab p' + sigma_ab
    energy    v_b (rhoE + p) + sum_a v_a sigma_ab - kappa dT/dx_b.

Pins: tests/test_oracle_3d.py (reduction to the pinned 2D oracle for data
invariant along x, along y and along z; cyclic axis symmetry; conservation;
hydrostatic balance; the ABC field is divergence free and a Beltrami field).
"""
import math

import torch

from . import DTYPE
from .physics import background


def pressure(q, z, P):
    rho, mx, my, mz, E = q
    ke = 0.5 * (mx * mx + my * my + mz * mz) / rho
    geo = rho * P.g * z if P.gravity else 0.0
    return (P.gamma - 1.0) * (E - ke - geo)


def fluxes(q, gx, gy, gz, z, P, heat_override=None):
    """Point-wise fluxes F (x), G (y), H (z) and the physical source S.

    q, gx, gy, gz: sequences of 5 tensors (the state and its x-, y- and
    z-derivatives); z: height.  heat_override: (Tx, Ty, Tz) replacing grad T
    in the heat flux (slip-wall boundary, Eq. 10).  Returns lists of 5."""
    rho, mx, my, mz, E = q
    grads = [gx, gy, gz]
    gm1 = P.gamma - 1.0
    g = P.g if P.gravity else 0.0
    m = [mx, my, mz]
    vel = [mx / rho, my / rho, mz / rho]
    kin = 0.5 * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2])
    p = gm1 * (E - rho * kin - rho * g * z)
    pbar, rhobar, _ = background(z, P)
    pprime = p - pbar
    T = p / (rho * P.R)
    # d[a][b] = d v_a / d x_b = (d m_a/d x_b - v_a d rho/d x_b) / rho
    d = [[(grads[b][1 + a] - vel[a] * grads[b][0]) / rho for b in range(3)] for a in range(3)]
    div = d[0][0] + d[1][1] + d[2][2]
    # d p / d x_b from the EOS; the z-derivative of rho g z adds rho g
    dp = []
    for b in range(3):
        gb = grads[b]
        s = gb[4] - (vel[0] * gb[1] + vel[1] * gb[2] + vel[2] * gb[3]) + kin * gb[0] - g * z * gb[0]
        if b == 2:
            s = s - rho * g
        dp.append(gm1 * s)
    dT = [(dp[b] - P.R * T * grads[b][0]) / (rho * P.R) for b in range(3)]
    if heat_override is not None:
        dT = list(heat_override)
    sigma = [[P.mu * ((2.0 / 3.0) * div * (1.0 if a == b else 0.0) - (d[a][b] + d[b][a])) for b in range(3)]
             for a in range(3)]
    out = []
    for b in range(3):
        f = [m[b]]
        for a in range(3):
            f.append(m[a] * vel[b] + (pprime if a == b else 0.0) + sigma[a][b])
        f.append(vel[b] * (E + p) + vel[0] * sigma[0][b] + vel[1] * sigma[1][b] + vel[2] * sigma[2][b]
                 - P.kappa * dT[b])
        out.append(f)
    zero = torch.zeros_like(rho)
    S = [zero, zero, zero, -g * (rho - rhobar) if P.gravity else zero, zero]
    return out[0], out[1], out[2], S


def wave_speed(q, z, nrm, h_normal, P):
    """|v.n| + c + 2 eta lambda_v, as the 2D reading R6."""
    rho, mx, my, mz, E = q
    p = pressure(q, z, P)
    c = torch.sqrt(P.gamma * p / rho)
    vn = (mx * nrm[0] + my * nrm[1] + mz * nrm[2]) / rho
    lam_v = max(4.0 / 3.0, P.gamma / P.Pr) * P.mu / rho
    eta = (2 * P.N + 1) / (h_normal * math.sqrt(math.pi / 2.0))
    return vn.abs() + c + 2.0 * eta * lam_v


def theta(q, z, P):
    """Potential temperature T (p0/p)^(R/c_p)."""
    p = pressure(q, z, P)
    T = p / (q[0] * P.R)
    return T * (P.p0 / p) ** (P.R / P.cp)


def abc_flow(x, y, z, t, P):
    """The ABC flow of Sec. 4.1 on [-pi, pi]^3: rho = 1,
    v = exp(-mu t) (sin z + cos y, sin x + cos z, sin y + cos x),
    p = -exp(-2 mu t) (cos x sin y + sin x cos z + sin z cos y) + 100/gamma."""
    t = torch.as_tensor(t, dtype=DTYPE)
    a = torch.exp(-P.mu * t)
    rho = 1.0 + 0.0 * x + 0.0 * y + 0.0 * z
    u = a * (torch.sin(z) + torch.cos(y))
    v = a * (torch.sin(x) + torch.cos(z))
    w = a * (torch.sin(y) + torch.cos(x))
    pr = (-torch.exp(-2.0 * P.mu * t) * (torch.cos(x) * torch.sin(y) + torch.sin(x) * torch.cos(z)
                                         + torch.sin(z) * torch.cos(y)) + 100.0 / P.gamma)
    E = pr / (P.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return [rho, rho * u, rho * v, rho * w, E]


def field_with_gradient(fn, x, y, z, t, P):
    """Q and its x-, y-, z-derivatives of an analytic field fn(x, y, z, t, P)
    by automatic differentiation (analytic boundary data)."""
    shape = x.shape
    xs = [c.reshape(-1).clone().requires_grad_(True) for c in (x, y, z)]
    with torch.enable_grad():
        Q = fn(xs[0], xs[1], xs[2], t, P)
        gs = [[], [], []]
        for c in Q:
            gr = torch.autograd.grad(c.sum(), xs, allow_unused=True, retain_graph=True)
            for b in range(3):
                gs[b].append((torch.zeros_like(xs[b]) if gr[b] is None else gr[b]).detach().reshape(shape))
    return [c.detach().reshape(shape) for c in Q], gs[0], gs[1], gs[2]


def cosine_bubble(x, y, z, A=0.5, a=250.0, xc=500.0, yc=500.0, zc=350.0):
    """Eq. 15 in 3D (Sec. 4.2: yc = xc): A/2 (1 + cos(pi r/a)) for r <= a."""
    r = torch.sqrt((x - xc) ** 2 + (y - yc) ** 2 + (z - zc) ** 2)
    return torch.where(r <= a, 0.5 * A * (1.0 + torch.cos(math.pi * r / a)), torch.zeros_like(r))


def bubble_state(z, theta_prime, P):
    """Background atmosphere with the temperature perturbed by theta' at the
    background pressure, at rest (the 2D reading of Sec. 4.2)."""
    pbar, _, _ = background(z, P)
    exner = 1.0 - P.g * z / (P.cp * P.theta0)
    T = (P.theta0 + theta_prime) * exner
    rho = pbar / (P.R * T)
    zero = torch.zeros_like(rho)
    E = pbar / (P.gamma - 1.0) + rho * P.g * z
    return [rho, zero, zero, zero, E]
