"""Batched persistent step of FP64 instances (the per-mesh FP64 predictor
and corrector bodies inside the persistent launches) against per-mesh FP64
steps and the FP64 oracle."""
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300.solver import (Batch, Mesh, atmosphere_config, cavity_config,
                                           paper_manufactured_config, steady_manufactured_config)
from tests.oracle_bridge import oracle_for
from tests.tolerances import momentum_floor

pytestmark = pytest.mark.gpu


def _bubble(side, radius, degree):
    m = Mesh(atmosphere_config(degree=degree, nx=side, ny=side))
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=radius, xc=500.0, zc=350.0)
    return m


def _close(a, b, tol, floor=0.0, what=""):
    """Per-variable L2: |a - b| <= tol |b| (+ floor on the momentum)."""
    a = a.detach().cpu().double()
    b = b.detach().cpu().double()
    for v in range(4):
        d = torch.linalg.vector_norm(a[:, v] - b[:, v]).item()
        nb = torch.linalg.vector_norm(b[:, v]).item()
        bound = tol * nb + (floor if v in (1, 2) else 0.0)
        assert d <= max(bound, 1e-300 * nb), f"{what} var {v}: |d|={d:.3e} |ref|={nb:.3e} bound={bound:.3e}"


@pytest.mark.parametrize("degree", [3, 5])
def test_fp64_batch_matches_individual_meshes(degree):
    """Bubbles on 5^2, 8^2, 11^2 cells: 3 then 2 graph-replayed batched steps
    against per-mesh FP64 steps.  Both run the same FP64 bodies with the same
    tile size; the compiler may contract a multiply-add differently in the
    two kernels, so the bound is 1e-13 relative plus the momentum floor of
    one rounding of p' per step."""
    sides, radii = (5, 8, 11), (300.0, 220.0, 150.0)
    a = [_bubble(s, r, degree) for s, r in zip(sides, radii)]
    b = [_bubble(s, r, degree) for s, r in zip(sides, radii)]
    dts = [m.stable_dt(0.25) for m in a]
    batch = Batch(a)
    info = batch.info()
    assert info["cpb_pred"] >= 1 and info["tiles_pred"] == sum(-(-s * s // info["cpb_pred"]) for s in sides)
    batch.step(dts, nsteps=3)
    batch.step(dts, nsteps=2)  # a new step count captures the graph again
    for m, dt in zip(b, dts):
        m.step(dt, 5)
    torch.cuda.synchronize()
    for ma, mb, dt in zip(a, b, dts):
        cfg = ma.cfg
        _close(ma.get_state(), mb.get_state(), 1e-13,
               momentum_floor(cfg, dt, 5, cfg.nx * cfg.ny * cfg.n ** 2), "batch vs mesh")
        assert abs(ma.time - mb.time) <= 1e-15 * mb.time
    batch.close()


def test_fp64_batch_mixed_scenarios_match_oracle():
    """One batch of three scenario kinds at degree 3 (a warm bubble with slip
    walls and gravity, the periodic steady manufactured case with its source,
    a no-slip lid-driven cavity), 6 steps each at its own dt: the first two
    against the FP64 oracle (1e-11 relative, the FP64 parity bound), the
    cavity against its per-mesh step."""
    bub = _bubble(9, 250.0, 3)
    man = Mesh(steady_manufactured_config(degree=3, nx=7, ny=7))
    man.init_scenario(L.ADG_SCEN_STEADY)
    cav = Mesh(cavity_config(degree=3, nx=6, ny=6))
    cav.init_scenario(L.ADG_SCEN_CAVITY)
    cav_ref = Mesh(cavity_config(degree=3, nx=6, ny=6))
    cav_ref.init_scenario(L.ADG_SCEN_CAVITY)
    ms = [bub, man, cav]
    dts = [bub.stable_dt(0.25), man.stable_dt(0.25), 0.5 * cav.stable_dt(0.25)]
    u0 = [m.get_state().cpu() for m in ms[:2]]
    batch = Batch(ms)
    batch.step(dts, nsteps=6)
    cav_ref.step(dts[2], 6)
    torch.cuda.synchronize()
    for m, u, dt in zip(ms[:2], u0, dts[:2]):
        o = oracle_for(m.cfg)
        uo = u
        for k in range(6):
            uo = o.step(uo, dt, k * dt)
        cfg = m.cfg
        _close(m.get_state(), uo, 1e-11, momentum_floor(cfg, dt, 6, cfg.nx * cfg.ny * cfg.n ** 2), "vs oracle")
    _close(cav.get_state(), cav_ref.get_state(), 1e-13, 0.0, "cavity batch vs mesh")
    batch.close()


def test_fp64_batch_rejections():
    fp = _bubble(5, 200.0, 3)
    mx = Mesh(atmosphere_config(degree=3, nx=5, ny=5, precision=L.ADG_PREC_MIXED))
    with pytest.raises(L.AdgError) as e:
        Batch([fp, mx])
    assert e.value.code == L.ADG_EINVAL
    tf = Mesh(atmosphere_config(degree=3, nx=5, ny=5, precision=L.ADG_PREC_MIXED_TF32))
    with pytest.raises(L.AdgError) as e:
        Batch([tf])
    assert e.value.code == L.ADG_EUNSUPPORTED
    paper = Mesh(paper_manufactured_config(degree=3, nx=5, ny=5))
    with pytest.raises(L.AdgError) as e:
        Batch([fp, paper])
    assert e.value.code == L.ADG_EUNSUPPORTED
    cfg = atmosphere_config(degree=3, nx=3, ny=3)
    cfg.max_levels = 1
    amr = Mesh(cfg)
    with pytest.raises(L.AdgError) as e:
        Batch([amr])
    assert e.value.code == L.ADG_EUNSUPPORTED
    batch = Batch([fp])
    with pytest.raises(L.AdgError) as e:
        batch.set_candidate(1)
    assert e.value.code == L.ADG_EUNSUPPORTED
    batch.close()
