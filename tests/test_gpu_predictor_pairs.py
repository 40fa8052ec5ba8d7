"""The node-pair mixed predictor (two nodes of a row per thread, degrees 3
and 5, the per-mesh launch) against the node-per-thread predictor (the
batched persistent launch's candidate 1 runs that body) and against the
batched node-pair kernel (candidate 3): the same arithmetic in the same
order on the same shared-memory layout, so the states agree bitwise (meshes
of several blocks with a ragged last block included)."""
import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.solver import Batch, Mesh, atmosphere_config, steady_manufactured_config

pytestmark = pytest.mark.gpu


def _bubble(degree, side, stir=True):
    m = Mesh(atmosphere_config(degree=degree, nx=side, ny=side, precision=L.ADG_PREC_MIXED))
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    if stir:  # momentum everywhere, so every flux term is active from the first step
        u = m.get_state().clone()
        pert = torch.from_numpy(inputs.perturbation(tuple(u[:, 1:3].shape), seed=degree, scale=0.5)).cuda()
        u[:, 1:3] += pert * u[:, 0:1]
        m.set_state(u)
    return m


@pytest.mark.parametrize("cand", [1, 3])
@pytest.mark.parametrize("degree,side", [(3, 13), (5, 9), (5, 13), (5, 14)])
def test_node_pairs_bitwise_equal_node_per_thread(degree, side, cand):
    a, b = _bubble(degree, side), _bubble(degree, side)
    dt = a.stable_dt(0.25)
    a.step(dt, 3)
    batch = Batch([b])
    batch.set_candidate(cand)
    batch.step([dt], nsteps=3)
    torch.cuda.synchronize()
    ua, ub = a.get_state(), b.get_state()
    assert torch.isfinite(ua).all()
    assert torch.equal(ua, ub), (ua - ub).abs().max().item()
    batch.close()
    a.close()
    b.close()


@pytest.mark.parametrize("cand", [1, 3])
@pytest.mark.parametrize("degree", [3, 5])
def test_node_pairs_steady_source_bitwise(degree, cand):
    """The steady manufactured source (x-dependent per node) on a periodic mesh."""
    cfg = steady_manufactured_config(degree=degree, nx=5, ny=4, precision=L.ADG_PREC_MIXED)
    a, b = Mesh(cfg), Mesh(cfg)
    a.init_scenario(L.ADG_SCEN_STEADY)
    b.init_scenario(L.ADG_SCEN_STEADY)
    dt = a.stable_dt(0.5)
    a.step(dt, 2)
    batch = Batch([b])
    batch.set_candidate(cand)
    batch.step([dt], nsteps=2)
    torch.cuda.synchronize()
    assert torch.equal(a.get_state(), b.get_state())
    batch.close()
    a.close()
    b.close()
