"""Point-wise physics of the compressible Navier-Stokes system (oracle).

Follows Sec. 2 of the paper:

* Eq. 1  conservative form Q = (rho, rho v, rho E), F = F^h(Q) + F^v(Q, grad Q),
         source S;
* Eq. 2  ideal-gas EOS with geopotential, p = (gamma-1)(rhoE - 1/2 v.rho v - rho g z)
         (reading: the printed "g z" is an energy per mass, so it is multiplied
         by rho -- rhoE is an energy density);
* Eq. 3  p = rho R T;
* Eq. 4  stress tensor sigma = mu((2/3) div v I - (grad v + grad v^T))
         (reading: the identity on the divergence term is implied);
* Eq. 5  heat coefficient kappa = mu gamma R / (Pr (gamma-1)) = mu c_p / Pr;
* Eq. 6  hydrostatic background d pbar/dz = -g rhobar;
* Eq. 7  perturbation split: the momentum flux carries p' = p - pbar(z) and
         the momentum source is -g k rho' with rho' = rho - rhobar(z);
* Sec. 4.2 potential temperature theta = T (p0/p)^(R/c_p), background from a
         constant potential temperature theta0 (isentropic atmosphere, Exner
         function pi(z) = 1 - g z/(c_p theta0)), cosine and Gaussian-tail
         bubbles (Eqs. 12-16; reading: cos(pi r / a) and r = |x - x_c|).

Gradients of primitive quantities are formed from grad Q by the chain rule.
With gravity off the background is zero, so p' = p.

Pins: tests/test_oracle_physics.py (autograd source of the steady manufactured
field equals its hand-derived closed form; background satisfies Eq. 6 to
rounding; theta of the initial bubble state equals theta0 + theta').
"""
import math
from dataclasses import dataclass, field

import torch

from . import DTYPE


@dataclass
class Params:
    N: int = 3
    gamma: float = 1.4
    Pr: float = 0.7
    R: float = 0.4            # c_v = R/(gamma-1) = 1 for the CFD scenarios
    mu: float = 0.1
    gravity: bool = False
    g: float = 9.81
    p0: float = 1e5
    theta0: float = 300.0
    source: str = "none"      # "none" | "steady" | "paper"
    man: dict = field(default_factory=dict)

    @property
    def cv(self):
        return self.R / (self.gamma - 1.0)

    @property
    def cp(self):
        return self.gamma * self.R / (self.gamma - 1.0)

    @property
    def kappa(self):
        return self.mu * self.gamma * self.R / (self.Pr * (self.gamma - 1.0))


def cfd_params(N, mu=0.1, source="steady"):
    """gamma = 1.4, Pr = 0.7, c_v = 1 (Sec. 4.1)."""
    return Params(N=N, gamma=1.4, Pr=0.7, R=0.4, mu=mu, gravity=False, source=source)


def atmosphere_params(N, mu=0.01, g=9.81):
    """gamma = 1.4, Pr = 0.71, R = 287.058, p0 = 1e5 Pa (Sec. 4.2, Eq. 11)."""
    return Params(N=N, gamma=1.4, Pr=0.71, R=287.058, mu=mu, gravity=True, g=g,
                  p0=1e5, theta0=300.0, source="none")


# ----------------------------------------------------------------- background
def background(z, P):
    """(pbar, rhobar, Tbar) of the isentropic atmosphere at height z; zero when
    gravity is off."""
    z = torch.as_tensor(z, dtype=DTYPE)
    if not P.gravity:
        zero = torch.zeros_like(z)
        return zero, zero, zero
    exner = 1.0 - P.g * z / (P.cp * P.theta0)
    Tbar = P.theta0 * exner
    pbar = P.p0 * exner ** (P.cp / P.R)
    rhobar = pbar / (P.R * Tbar)
    return pbar, rhobar, Tbar


def dTbar_dz(P):
    """Background temperature gradient (constant for the isentropic profile)."""
    return -P.g / P.cp if P.gravity else 0.0


# -------------------------------------------------------------------- fluxes
def pressure(q, z, P):
    rho, mx, my, E = q
    ke = 0.5 * (mx * mx + my * my) / rho
    geo = rho * P.g * z if P.gravity else 0.0
    return (P.gamma - 1.0) * (E - ke - geo)


def fluxes(q, qx, qy, z, P, heat_override=None):
    """Point-wise F (x-flux), G (y-flux) and physical source S.

    q, qx, qy: sequences of 4 tensors (rho, rho u, rho v, rho E) and their x-
    and y-derivatives, all of one broadcastable shape; z: height (= y).
    heat_override: if given, (Tx, Ty) replaces grad T in the heat flux (the
    wall boundary condition Eq. 10 imposes the background heat flux).
    Returns F, G, S as lists of 4 tensors.
    """
    rho, mx, my, E = q
    rx, mxx, myx, Ex = qx
    ry, mxy, myy, Ey = qy
    gm1 = P.gamma - 1.0
    u = mx / rho
    v = my / rho
    g = P.g if P.gravity else 0.0
    p = gm1 * (E - 0.5 * (mx * u + my * v) - rho * g * z)
    pbar, rhobar, _ = background(z, P)
    pprime = p - pbar
    rhoprime = rho - rhobar
    T = p / (rho * P.R)
    # velocity gradients by the chain rule: grad v = (grad(rho v) - v grad rho)/rho
    ux = (mxx - u * rx) / rho
    uy = (mxy - u * ry) / rho
    vx = (myx - v * rx) / rho
    vy = (myy - v * ry) / rho
    # grad p from the EOS (z-derivative of rho g z contributes rho g)
    kin = 0.5 * (u * u + v * v)
    px = gm1 * (Ex - (u * mxx + v * myx) + kin * rx - g * z * rx)
    py = gm1 * (Ey - (u * mxy + v * myy) + kin * ry - g * z * ry - rho * g)
    # grad T from p = rho R T
    Tx = (px - P.R * T * rx) / (rho * P.R)
    Ty = (py - P.R * T * ry) / (rho * P.R)
    if heat_override is not None:
        Tx, Ty = heat_override
    div = ux + vy
    sxx = P.mu * ((2.0 / 3.0) * div - 2.0 * ux)
    syy = P.mu * ((2.0 / 3.0) * div - 2.0 * vy)
    sxy = -P.mu * (uy + vx)
    k = P.kappa
    F = [mx,
         mx * u + pprime + sxx,
         my * u + sxy,
         u * (E + p) + u * sxx + v * sxy - k * Tx]
    G = [my,
         mx * v + sxy,
         my * v + pprime + syy,
         v * (E + p) + u * sxy + v * syy - k * Ty]
    zero = torch.zeros_like(rho)
    S = [zero, zero, -g * rhoprime if P.gravity else zero, zero]
    return F, G, S


def wave_speed(q, z, nx, ny, h_normal, P):
    """Rusanov speed of a face state: |v.n| + c + 2 eta lambda_v with
    lambda_v = max(4/3, gamma/Pr) mu/rho and eta = (2N+1)/(h sqrt(pi/2))
    (viscous Rusanov flux of Gassner et al. 2008 as used with ADER-DG by
    Dumbser 2010; the paper cites both but prints no constant: parity
    unpinned for the constant)."""
    rho, mx, my, E = q
    p = pressure(q, z, P)
    c = torch.sqrt(P.gamma * p / rho)
    vn = (mx * nx + my * ny) / rho
    lam_v = max(4.0 / 3.0, P.gamma / P.Pr) * P.mu / rho
    eta = (2 * P.N + 1) / (h_normal * math.sqrt(math.pi / 2.0))
    return vn.abs() + c + 2.0 * eta * lam_v


def theta(q, z, P):
    """Potential temperature theta = T (p0/p)^(R/c_p) (Sec. 4.2)."""
    p = pressure(q, z, P)
    T = p / (q[0] * P.R)
    return T * (P.p0 / p) ** (P.R / P.cp)


# ------------------------------------------------------------ scenario fields
def steady_manufactured(x, y, t, P, a=0.1, L=10.0, U=0.5, p=1.0):
    """rho = 1 + a sin(2 pi (x+y)/L), u = v = U, p = const (time independent)."""
    rho = 1.0 + a * torch.sin(2.0 * math.pi * (x + y) / L) + 0.0 * t
    u = U + 0.0 * rho
    v = U + 0.0 * rho
    pr = p + 0.0 * rho
    E = pr / (P.gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return [rho, rho * u, rho * v, E]


def paper_manufactured(x, y, t, P):
    """Eq. 8: p = cos(phi)/10 + 1/gamma, rho = sin(phi)/2 + 1,
    v = (1,1) sin(phi)/4 with phi = pi/5 (x + y) - 2 pi t."""
    phi = math.pi / 5.0 * (x + y) - 2.0 * math.pi * t
    pr = 0.1 * torch.cos(phi) + 1.0 / P.gamma
    rho = 0.5 * torch.sin(phi) + 1.0
    u = 0.25 * torch.sin(phi)
    v = 0.25 * torch.sin(phi)
    E = pr / (P.gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return [rho, rho * u, rho * v, E]


def taylor_green(x, y, t, P):
    """The Taylor-Green vortex of Sec. 4.1 (incompressible form, imposed as
    initial and boundary data): rho = 1, v = exp(-2 mu t) (sin x cos y,
    -cos x sin y), p = exp(-4 mu t) (cos 2x + cos 2y) / 4 + 100/gamma."""
    t = torch.as_tensor(t, dtype=DTYPE)
    a = torch.exp(-2.0 * P.mu * t)
    rho = 1.0 + 0.0 * x + 0.0 * y
    u = a * torch.sin(x) * torch.cos(y)
    v = -a * torch.cos(x) * torch.sin(y)
    pr = torch.exp(-4.0 * P.mu * t) * 0.25 * (torch.cos(2.0 * x) + torch.cos(2.0 * y)) + 100.0 / P.gamma
    E = pr / (P.gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return [rho, rho * u, rho * v, E]


def field_with_gradient(fn, x, y, t, P):
    """Q, dQ/dx, dQ/dy of an analytic field fn(x, y, t, P) by automatic
    differentiation (for Dirichlet boundary data)."""
    shape = x.shape
    x = x.reshape(-1).clone().requires_grad_(True)
    y = y.reshape(-1).clone().requires_grad_(True)
    with torch.enable_grad():
        Q = fn(x, y, t, P)
        qx, qy = [], []
        for c in Q:
            gx, gy = torch.autograd.grad(c.sum(), [x, y], allow_unused=True, retain_graph=True)
            qx.append((torch.zeros_like(x) if gx is None else gx).detach().reshape(shape))
            qy.append((torch.zeros_like(y) if gy is None else gy).detach().reshape(shape))
    return [c.detach().reshape(shape) for c in Q], qx, qy


def manufactured_field(P):
    return {"steady": steady_manufactured, "paper": paper_manufactured}[P.source]


def manufactured_source(x, y, t, P):
    """S = dQ/dt + dF/dx + dG/dy - S_phys(Q) for the analytic field, by
    automatic differentiation of the field and of `fluxes` (the definition
    of a manufactured source, Sec. 4.1)."""
    field_fn = manufactured_field(P)
    shape = x.shape
    x = x.reshape(-1).clone().requires_grad_(True)
    y = y.reshape(-1).clone().requires_grad_(True)
    t = torch.as_tensor(t, dtype=DTYPE).expand_as(x).clone().requires_grad_(True)
    with torch.enable_grad():
        Q = field_fn(x, y, t, P)
        Qx, Qy, Qt = [], [], []
        for c in Q:
            gx, gy, gt = torch.autograd.grad(c.sum(), [x, y, t], create_graph=True)
            Qx.append(gx)
            Qy.append(gy)
            Qt.append(gt)
        F, G, Sp = fluxes(Q, Qx, Qy, y, P)
        out = []
        for v in range(4):
            dFx = torch.autograd.grad(F[v].sum(), x, retain_graph=True, allow_unused=True)[0]
            dGy = torch.autograd.grad(G[v].sum(), y, retain_graph=True, allow_unused=True)[0]
            dFx = torch.zeros_like(x) if dFx is None else dFx
            dGy = torch.zeros_like(x) if dGy is None else dGy
            out.append((Qt[v] + dFx + dGy - Sp[v]).detach().reshape(shape))
    return out


def bubble_state(x, z, theta_prime, P):
    """Conserved state of the background atmosphere perturbed by theta'
    (reading of Sec. 4.2: pressure stays at the background, the temperature
    carries the perturbation, the fluid is at rest)."""
    pbar, _, _ = background(z, P)
    exner = 1.0 - P.g * z / (P.cp * P.theta0)
    T = (P.theta0 + theta_prime) * exner
    rho = pbar / (P.R * T)
    zero = torch.zeros_like(rho)
    E = pbar / (P.gamma - 1.0) + rho * P.g * z
    return [rho, zero, zero, E]


def cosine_bubble(x, z, A=0.5, a=250.0, xc=500.0, zc=350.0):
    """Eq. 15 (reading: cos(pi r / a), r = Euclidean distance to the centre)."""
    r = torch.sqrt((x - xc) ** 2 + (z - zc) ** 2)
    return torch.where(r <= a, 0.5 * A * (1.0 + torch.cos(math.pi * r / a)), torch.zeros_like(r))


def gaussian_bubble(x, z, A, a, s, xc, zc):
    """Eq. 12: A for r <= a, A exp(-(r-a)^2/s^2) beyond."""
    r = torch.sqrt((x - xc) ** 2 + (z - zc) ** 2)
    return torch.where(r <= a, A + 0.0 * r, A * torch.exp(-((r - a) ** 2) / (s * s)))


def two_bubbles(x, z):
    """Eq. 14 values: warm (0.5 K, a=150, s=50, (500,300)) plus cold
    (-0.15 K, a=0, s=50, (560,640)); theta' is their sum."""
    return (gaussian_bubble(x, z, 0.5, 150.0, 50.0, 500.0, 300.0)
            + gaussian_bubble(x, z, -0.15, 0.0, 50.0, 560.0, 640.0))
