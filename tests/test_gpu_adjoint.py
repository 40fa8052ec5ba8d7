"""Hand-written discrete adjoint of one FP64 step (adg_step_adjoint) against
the oracle's discrete adjoint (reverse-mode differentiation of the oracle
step) and against central finite differences of the GPU forward step."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.solver import Mesh, MeshConfig, atmosphere_config, steady_manufactured_config
from tests.oracle_bridge import oracle_for, steady_field, cosine_field

pytestmark = pytest.mark.gpu


def gpu_adjoint(m, dt, u, lam):
    out = torch.empty_like(lam)
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(m._lib.adg_step_adjoint(m.h, float(dt), ctypes.c_void_p(u.data_ptr()),
                                    ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(out.data_ptr()), sp))
    torch.cuda.synchronize()
    return out


def oracle_adjoint(o, dt, u, lam):
    u = u.clone().requires_grad_(True)
    with torch.enable_grad():
        y = o.step(u, dt)
        (g,) = torch.autograd.grad(y, u, grad_outputs=lam)
    return g


def rel(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


CASES = [
    ("steady N=1 5x4", lambda: steady_manufactured_config(degree=1, nx=5, ny=4)),
    ("steady N=2 5x4", lambda: steady_manufactured_config(degree=2, nx=5, ny=4)),
    ("steady N=3 3x3", lambda: steady_manufactured_config(degree=3, nx=3, ny=3)),
    ("bubble N=3 9x9", lambda: atmosphere_config(degree=3, nx=9, ny=9)),
    ("bubble N=4 5x5", lambda: atmosphere_config(degree=4, nx=5, ny=5)),
    ("bubble N=5 4x3", lambda: atmosphere_config(degree=5, nx=4, ny=3)),
]


@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_oracle(name, mk):
    cfg = mk()
    o = oracle_for(cfg)
    if cfg.gravity:
        u0 = cosine_field(o)
        # a seeded velocity field so that the flow is not at rest
        mom = torch.from_numpy(inputs.perturbation((cfg.cells, 2, cfg.n, cfg.n), seed=21, scale=0.5))
        u0 = u0.clone()
        u0[:, 1:3] += mom * u0[:, 0:1]
    else:
        u0 = steady_field(o, cfg)
        u0 = u0 + torch.from_numpy(inputs.perturbation(tuple(u0.shape), seed=22, scale=1e-2))
    dt = o.stable_dt(u0, 0.25)
    lam = torch.from_numpy(inputs.perturbation(tuple(u0.shape), seed=23, scale=1.0))
    g_or = oracle_adjoint(o, dt, u0, lam)
    m = Mesh(cfg)
    g_gpu = gpu_adjoint(m, dt, u0.cuda().contiguous(), lam.cuda().contiguous()).cpu()
    r = rel(g_gpu, g_or)
    assert r <= 1e-10, (name, r)


def test_adjoint_directional_derivative_fd():
    """<lam_n, d> equals the central difference of <lam', step(u)> along d."""
    cfg = atmosphere_config(degree=3, nx=9, ny=9)
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    dt = m.stable_dt(0.25)
    u0 = m.get_state().clone()
    lam = torch.from_numpy(inputs.perturbation(tuple(u0.shape), seed=31, scale=1.0)).cuda()
    g = gpu_adjoint(m, dt, u0, lam)
    for seed in range(4):
        d = torch.from_numpy(inputs.perturbation(tuple(u0.shape), seed=40 + seed, scale=1.0)).cuda()
        d = d * u0.abs().amax(dim=(0, 2, 3), keepdim=True) * 1e-3   # scale per variable
        h = 1e-4

        def J(x):
            m.set_state(x.contiguous())
            m.step(dt)
            return float((lam * m.get_state()).sum())

        fd = (J(u0 + h * d) - J(u0 - h * d)) / (2 * h)
        ad = float((g * d).sum())
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-30), (seed, fd, ad)


def test_adjoint_rejects_mixed_and_aliasing():
    cfg = atmosphere_config(degree=3, nx=3, ny=3, precision=L.ADG_PREC_MIXED)
    m = Mesh(cfg)
    u = torch.zeros(m.count, dtype=torch.float64, device="cuda")
    with pytest.raises(L.AdgError) as e:
        gpu_adjoint(m, 0.01, u, u.clone())
    assert e.value.code == L.ADG_EUNSUPPORTED
