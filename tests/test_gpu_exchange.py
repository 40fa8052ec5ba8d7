"""Strip decomposition on the GPU library (bc_y = ADG_BC_EXCHANGE*): two strip
meshes on one device, their edge traces exchanged by device copies exactly as
exchange.StripStepper does between ranks, reproduce the single-mesh step;
per-strip statistics combined with Chan's update reproduce the global flags."""
import ctypes

import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.exchange import LibraryStrip, combine_stats, strip_bc, strip_rows
from paper_1905_05524_gb300.solver import Mesh, MeshConfig, atmosphere_config
from tests.tolerances import momentum_floor

pytestmark = pytest.mark.gpu


def _strips(cfg, world, periodic):
    out = []
    hy = cfg.Ly / cfg.ny
    for r in range(world):
        first, rows = strip_rows(cfg.ny, world, r)
        c = MeshConfig(**{**cfg.__dict__})
        c.ny, c.y0, c.Ly = rows, cfg.y0 + first * hy, rows * hy
        c.bc_y = strip_bc(r, world, periodic)
        out.append((first, rows, LibraryStrip(Mesh(c))))
    return out


def _run(cfg, u0, dt, steps, periodic, world=2):
    strips = _strips(cfg, world, periodic)
    nx = cfg.nx
    for first, rows, b in strips:
        b.m.set_state(u0[first * nx:(first + rows) * nx].contiguous())
    for _ in range(steps):
        for _, _, b in strips:
            b.predictor(dt)
        tr = [tuple(t.clone() for t in b.boundary_traces()) for _, _, b in strips]
        for r, (_, _, b) in enumerate(strips):
            below = r - 1 if r > 0 else (world - 1 if periodic else None)
            above = r + 1 if r < world - 1 else (0 if periodic else None)
            b.set_halo(tr[below][1] if below is not None else None, tr[above][0] if above is not None else None)
        for _, _, b in strips:
            b.corrector(dt)
    return torch.cat([b.m.get_state() for _, _, b in strips], 0), strips


def test_periodic_strips_equal_single_mesh_bitwise():
    cfg = MeshConfig(degree=3, nx=7, ny=8, mu=0.05)
    g = Mesh(cfg)
    u0 = (1.0 + torch.from_numpy(inputs.perturbation((56, 4, 4, 4), seed=2, scale=0.05))).cuda()
    u0[:, 3] += 2.0
    g.set_state(u0.contiguous())
    g.step(0.01, 4)
    full, _ = _run(cfg, u0, 0.01, 4, periodic=True)
    assert torch.equal(full, g.get_state())


def test_walled_bubble_strips_match_single_mesh():
    cfg = atmosphere_config(degree=5, nx=9, ny=9)
    g = Mesh(cfg)
    g.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    u0 = g.get_state().clone()
    dt = g.stable_dt(0.25)
    g.step(dt, 5)
    ref = g.get_state()
    for world in (2, 3):
        full, strips = _run(cfg, u0, dt, 5, periodic=False, world=world)
        floor = momentum_floor(cfg, dt, 5, ref[:, 0].numel())
        for v in range(4):
            d = torch.linalg.vector_norm(full[:, v] - ref[:, v]).item()
            bound = 1e-11 * torch.linalg.vector_norm(ref[:, v]).item() + (floor if v in (1, 2) else 0.0)
            assert d <= bound, (world, v, d, bound)
        # global refinement flags from per-strip statistics combined by Chan's update
        tvs, trip = [], []
        for _, _, b in strips:
            tv, _, (mean, std) = b.m.tv_indicator(L.ADG_TV_THETA, 1.5, -0.5)
            tvs.append(tv)
            trip.append((b.m.leaves, mean, std * std * b.m.leaves))
        cnt, mean, m2 = combine_stats(trip)
        tvg, flg, (mg, sg) = g.tv_indicator(L.ADG_TV_THETA, 1.5, -0.5)
        assert abs(mean - mg) <= 1e-9 * abs(mg) and abs((m2 / cnt) ** 0.5 - sg) <= 1e-9 * sg
        fl = []
        for tv, (_, _, b) in zip(tvs, strips):
            f = torch.empty(b.m.leaves, dtype=torch.int8, device="cuda")
            L.check(b.m._lib.adg_tv_flags(b.m.h, ctypes.c_void_p(tv.data_ptr()), float(cnt), float(mean), float(m2),
                                          1.5, -0.5, ctypes.c_void_p(f.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
            fl.append(f)
        assert torch.equal(torch.cat(fl), flg)
