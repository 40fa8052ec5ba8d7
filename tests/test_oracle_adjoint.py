"""Pin of the oracle's discrete adjoint (reverse-mode differentiation of the
oracle step) against central finite differences of the oracle step."""
import torch

from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.solver import atmosphere_config
from tests.oracle_bridge import oracle_for, cosine_field


def _vjp(o, dt, u, lam):
    u = u.clone().requires_grad_(True)
    with torch.enable_grad():
        y = o.step(u, dt)
        (g,) = torch.autograd.grad(y, u, grad_outputs=lam)
    return g


def test_oracle_adjoint_matches_central_differences():
    cfg = atmosphere_config(degree=2, nx=4, ny=4)
    o = oracle_for(cfg)
    u0 = cosine_field(o)
    u0[:, 1:3] += torch.from_numpy(inputs.perturbation((16, 2, 3, 3), seed=5, scale=0.5)) * u0[:, 0:1]
    dt = o.stable_dt(u0, 0.25)
    lam = torch.from_numpy(inputs.perturbation(tuple(u0.shape), seed=6, scale=1.0))
    g = _vjp(o, dt, u0, lam)
    scale = u0.abs().amax(dim=(0, 2, 3), keepdim=True)
    for seed in range(6):
        d = torch.from_numpy(inputs.perturbation(tuple(u0.shape), seed=60 + seed, scale=1.0)) * scale * 1e-3
        h = 1e-4
        fd = ((lam * o.step(u0 + h * d, dt)).sum() - (lam * o.step(u0 - h * d, dt)).sum()) / (2 * h)
        ad = (g * d).sum()
        assert abs(fd - ad) <= 1e-6 * abs(ad), (seed, float(fd), float(ad))
