"""Batched persistent, graph-captured step of many independent instances
against per-instance steps (same kernels' arithmetic) and the FP64 oracle."""
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.solver import Batch, Mesh, atmosphere_config, steady_manufactured_config
from tests.oracle_bridge import oracle_for, cosine_field
from oracle import physics as ph

pytestmark = pytest.mark.gpu


def _bubble_mesh(side, radius, prec=L.ADG_PREC_MIXED, degree=5):
    cfg = atmosphere_config(degree=degree, nx=side, ny=side, precision=prec)
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=radius, xc=500.0, zc=350.0)
    return m


def _same(a, b, tol=1e-12):
    """Per-variable relative L2 <= tol (momentum floored at 1 m/s): the
    batched kernels run the per-mesh kernel body; they may differ in the
    last FP32 bits of the contractions, never more."""
    for v in range(4):
        d = torch.linalg.vector_norm(a[:, v] - b[:, v]).item()
        nb = torch.linalg.vector_norm(b[:, v]).item()
        den = max(nb, torch.linalg.vector_norm(b[:, 0]).item()) if v in (1, 2) else nb
        assert d <= tol * den, (v, d, den)


def test_batch_matches_individual_meshes():
    """Instances of uneven sizes (seeded sides 9..30, radii 100..300 m):
    3 graph-replayed batched steps equal 3 per-mesh steps."""
    sides = inputs.instance_sizes(5, seed=3, lo=9, hi=30)
    radii = inputs.uniform_values(5, seed=4, lo=100.0, hi=300.0)
    a = [_bubble_mesh(int(s), float(r)) for s, r in zip(sides, radii)]
    b = [_bubble_mesh(int(s), float(r)) for s, r in zip(sides, radii)]
    dts = [m.stable_dt(0.25) for m in a]
    batch = Batch(a)
    info = batch.info()
    assert info["tiles_pred"] > 0 and info["cpb_pred"] >= 1
    batch.step(dts, nsteps=3)
    for m, dt in zip(b, dts):
        m.step(dt, 3)
    torch.cuda.synchronize()
    for ma, mb in zip(a, b):
        _same(ma.get_state(), mb.get_state())
    # replay with a new step count re-captures the graph
    batch.step(dts, nsteps=2)
    for m, dt in zip(b, dts):
        m.step(dt, 2)
    for ma, mb in zip(a, b):
        _same(ma.get_state(), mb.get_state())
    batch.close()


def test_batch_vs_oracle_theta():
    """Two batched instances, 10 steps, theta' within 1e-6 of the FP64 oracle."""
    ms = [_bubble_mesh(9, 250.0, degree=3), _bubble_mesh(12, 180.0, degree=3)]
    dts = [m.stable_dt(0.25) for m in ms]
    u0 = [m.get_state().cpu() for m in ms]
    batch = Batch(ms)
    batch.step(dts, nsteps=10)
    for m, u, dt in zip(ms, u0, dts):
        o = oracle_for(m.cfg)
        uo = u
        for _ in range(10):
            uo = o.step(uo, dt)
        a = m.get_state().cpu()
        ta = ph.theta(a.unbind(1), o.Y, o.P) - o.P.theta0
        tb = ph.theta(uo.unbind(1), o.Y, o.P) - o.P.theta0
        assert (torch.linalg.vector_norm(ta - tb) / torch.linalg.vector_norm(tb)).item() <= 1e-6
    batch.close()


def test_batch_rejects_mixed_degrees_and_precisions():
    m1 = _bubble_mesh(9, 200.0, degree=3)
    m2 = _bubble_mesh(9, 200.0, degree=4)
    with pytest.raises(L.AdgError):
        Batch([m1, m2])
    m3 = _bubble_mesh(9, 200.0, prec=L.ADG_PREC_FP64, degree=3)
    with pytest.raises(L.AdgError) as e:
        Batch([m1, m3])
    assert e.value.code == L.ADG_EINVAL


@pytest.mark.parametrize("degree", [1, 2, 4, 6, 7])
def test_batch_matches_individual_meshes_every_degree(degree):
    """Three small instances (sides 5, 8, 11) per degree, 2 batched steps
    against 2 per-mesh steps: every tile-size candidate the autotuner may
    pick runs the per-mesh kernel body.  A candidate other than the
    per-mesh tile size is a separate instantiation whose FP32 rounding may
    differ in the last bits: 1e-9 relative (FP32 perturbations of ~1e-3 of
    the state)."""
    a = [_bubble_mesh(s, 300.0, degree=degree) for s in (5, 8, 11)]
    b = [_bubble_mesh(s, 300.0, degree=degree) for s in (5, 8, 11)]
    dts = [m.stable_dt(0.25) for m in a]
    batch = Batch(a)
    batch.step(dts, nsteps=2)
    for m, dt in zip(b, dts):
        m.step(dt, 2)
    torch.cuda.synchronize()
    for ma, mb in zip(a, b):
        _same(ma.get_state(), mb.get_state(), 1e-9)
    batch.close()


@pytest.mark.parametrize("degree", [2, 3, 5, 7])
@pytest.mark.parametrize("cand", [0, 1, 2, 3])
def test_batch_every_tile_candidate_matches_individual_meshes(degree, cand):
    """Each predictor candidate pinned in turn (half, default and double the
    per-mesh cells per block: separate instantiations of the slice-pair
    predictor body with their own shared-memory strides; 3: the node-pair
    body at degrees 3 and 5, candidate 1 elsewhere), 2 batched steps against
    2 per-mesh steps; 1e-9 relative as above (the default candidate is the
    per-mesh kernel's own tile size)."""
    a = [_bubble_mesh(s, 300.0, degree=degree) for s in (5, 8, 11)]
    b = [_bubble_mesh(s, 300.0, degree=degree) for s in (5, 8, 11)]
    dts = [m.stable_dt(0.25) for m in a]
    batch = Batch(a)
    batch.set_candidate(cand)
    info = batch.info()
    assert info["cpb_pred"] >= 1 and info["tiles_pred"] >= 1
    batch.step(dts, nsteps=2)
    for m, dt in zip(b, dts):
        m.step(dt, 2)
    torch.cuda.synchronize()
    for ma, mb in zip(a, b):
        _same(ma.get_state(), mb.get_state(), 1e-9)
    batch.close()
