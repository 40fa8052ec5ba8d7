"""Adaptive meshes inside the batched persistent, graph-captured launch
(Sec. 3's dynamic AMR with the batch of independent instances): the leaves of
every level of an adaptive instance and the cells of uniform instances run in
the same persistent predictor and corrector launches.  Checked against the
per-mesh adaptive kernels (the same bodies: bitwise), after an adaptation of
a member (the batch rebuilds its tables and graph), against the oracle's tree,
and the tuner's JSON cache across processes."""
import json
import os
import subprocess
import sys

import pytest
import torch

from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300.solver import Batch, Mesh, atmosphere_config
from oracle.amr import AmrSolver
from oracle import physics as ph

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _two_bubble_tree(degree=5, nx=27, levels=2):
    """The two-bubble initial mesh procedure (init -> TV -> refine, repeated,
    re-initialising from the analytic field), mixed precision."""
    cfg = atmosphere_config(degree=degree, nx=nx, ny=nx, mu=0.001, precision=L.ADG_PREC_MIXED)
    cfg.max_levels = levels
    m = Mesh(cfg)
    m.init_scenario(L.ADG_SCEN_TWO_BUBBLES)
    for _ in range(levels):
        _, fl, _ = m.tv_indicator(L.ADG_TV_THETA, 2.5, -0.5)
        m.adapt(torch.where(fl > 0, 1, 0).to(torch.int8))
        m.init_scenario(L.ADG_SCEN_TWO_BUBBLES)
    return m


def _bubble(side, degree=5):
    m = Mesh(atmosphere_config(degree=degree, nx=side, ny=side, precision=L.ADG_PREC_MIXED))
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    return m


def _twins(degree=5):
    a = [_two_bubble_tree(degree), _bubble(9, degree), _bubble(13, degree)]
    b = [_two_bubble_tree(degree), _bubble(9, degree), _bubble(13, degree)]
    assert a[0].leaf_info() == b[0].leaf_info() and len({c[0] for c in a[0].leaf_info()}) >= 2
    dts = [m.stable_dt(0.25) for m in a]
    return a, b, dts


@pytest.mark.parametrize("degree", [3, 5])
def test_adaptive_instance_in_batch_bitwise_per_mesh(degree):
    a, b, dts = _twins(degree)
    batch = Batch(a)
    batch.set_candidate(1)           # the per-mesh kernels' cells per block
    info = batch.info()
    assert info["adaptive_instances"] == 1
    assert info["tiles_pred"] >= sum(-(-m.leaves // info["cpb_pred"]) for m in a)
    batch.step(dts, nsteps=3)
    for m, dt in zip(b, dts):
        m.step(dt, 3)
    torch.cuda.synchronize()
    for ma, mb in zip(a, b):
        assert torch.isfinite(ma.get_state()).all()
        assert torch.equal(ma.get_state(), mb.get_state())
    batch.close()


def test_batch_rebuilds_after_adapt():
    """Two batched steps, an adaptation of the adaptive member (TV flags,
    refine and coarsen), two more batched steps: the batch picks up the new
    leaves and moved state (tables, tiles and graph rebuilt) and still equals
    the per-mesh run bitwise."""
    a, b, dts = _twins(5)
    batch = Batch(a)
    batch.set_candidate(1)
    batch.step(dts, nsteps=2)
    for m, dt in zip(b, dts):
        m.step(dt, 2)
    leaves0 = a[0].leaves
    for m in (a[0], b[0]):
        _, fl, _ = m.tv_indicator(L.ADG_TV_THETA, 1.0, -0.5)
        m.adapt(fl.contiguous())
    assert a[0].leaves == b[0].leaves and a[0].leaves != leaves0
    dts2 = [a[0].stable_dt(0.25)] + dts[1:]
    batch.step(dts2, nsteps=2)
    for m, dt in zip(b, dts2):
        m.step(dt, 2)
    torch.cuda.synchronize()
    for ma, mb in zip(a, b):
        assert torch.equal(ma.get_state(), mb.get_state())
    batch.close()


def test_batched_two_bubble_tree_step_vs_oracle():
    """One batched step of the two-bubble adaptive instance (27x27 base, two
    levels) against the oracle's tree: theta' within the mixed bound 1e-6
    and total rho within 1e-9."""
    m = _two_bubble_tree(5)
    P = ph.atmosphere_params(5, mu=0.001)
    o = AmrSolver(27, 27, P, 1000.0, 1000.0, bc="wall", max_level=2)
    o.leaves = [tuple(c) for c in m.leaf_info()]
    o._index()
    X, Y = o.node_coords()
    u = torch.stack(ph.bubble_state(X, Y, ph.two_bubbles(X, Y), P), 1)
    dt = m.stable_dt(0.25)
    uo = o.step(u, dt)
    batch = Batch([m, _bubble(9)])
    batch.step([dt, dt], nsteps=1)
    a = m.get_state().cpu()
    ta = ph.theta(a.unbind(1), Y, P) - P.theta0
    tb = ph.theta(uo.unbind(1), Y, P) - P.theta0
    assert (torch.linalg.vector_norm(ta - tb) / torch.linalg.vector_norm(tb)).item() <= 1e-6
    assert (torch.linalg.vector_norm(a[:, 0] - uo[:, 0]) / torch.linalg.vector_norm(uo[:, 0])).item() <= 1e-9
    batch.close()


_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import torch
from paper_1905_05524_gb300 import _lib as L
from paper_1905_05524_gb300.solver import Batch, Mesh, atmosphere_config
ms = []
for side in (7, 10):
    m = Mesh(atmosphere_config(degree=2, nx=side, ny=side, precision=L.ADG_PREC_MIXED))
    m.init_scenario(L.ADG_SCEN_COSINE, A=0.5, a=250.0, xc=500.0, zc=350.0)
    ms.append(m)
b = Batch(ms)
print(json.dumps(b.info()))
"""


def test_tuner_json_cache_across_processes(tmp_path):
    """The first process times the candidates and writes the JSON cache; a
    second process with the same cache file takes the choice from it."""
    cache = tmp_path / "tune.json"
    env = dict(os.environ, ADG_TUNE_CACHE=str(cache))
    runs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], env=env, capture_output=True, text=True,
                           timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        runs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    entries = json.loads(cache.read_text())
    assert any(e["key"].startswith("degree=2 precision=mixed") for e in entries)
    assert runs[0]["tune_source"] == 0 and runs[1]["tune_source"] == 2
    assert runs[0]["candidate"] == runs[1]["candidate"]
