"""Multi-rank paths on CPU ranks over gloo (world size 2): the strip
decomposition with one face-trace exchange per step (oracle backend) equals
the single-domain step, Chan's combination of per-rank statistics equals the
global statistics, and bench.py's max-over-ranks timing reduction."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1905_05524_gb300 import inputs
from paper_1905_05524_gb300.exchange import (StripStepper, combine_stats, gather_stats, strip_rows, exchange_halos)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _strip_worker(rank, world, port, case, out):
    _init(rank, world, port)
    try:
        from oracle import physics as ph
        from oracle.aderdg import Mesh, Solver
        from tests.oracle_strip import OracleStrip
        if case == "periodic":
            P = ph.cfd_params(2, mu=0.05, source="none")
            nx, ny, Lx, Ly, bc = 5, 7, 10.0, 10.0, "periodic"
            g = Solver(Mesh(nx, ny, Lx=Lx, Ly=Ly), P)
            u0 = g.interpolate(ph.steady_manufactured)
            u0 = u0 + torch.from_numpy(inputs.perturbation(tuple(u0.shape), seed=9, scale=1e-2))
        else:
            P = ph.atmosphere_params(2)
            nx, ny, Lx, Ly, bc = 5, 6, 1000.0, 1000.0, "wall"
            g = Solver(Mesh(nx, ny, Lx=Lx, Ly=Ly, bc_x="wall", bc_y="wall"), P)
            th = ph.cosine_bubble(g.X, g.Y)
            u0 = torch.stack(ph.bubble_state(g.X, g.Y, th, P), 1)
        dt = g.stable_dt(u0, 0.25)
        first, rows = strip_rows(ny, world, rank)
        if bc == "periodic":
            sbc = "halo"
        else:
            sbc = "wall_halo" if rank == 0 else ("halo_wall" if rank == world - 1 else "halo")
        mine = u0[first * nx:(first + rows) * nx].clone()
        strip = OracleStrip(P, nx, rows, first, ny, Lx, Ly, 0.0, sbc, mine)
        if bc == "wall":
            strip.s.m.bc_x = "wall"
        stepper = StripStepper(strip, rank, world, periodic=(bc == "periodic"))
        for _ in range(3):
            stepper.step(dt)
        parts = [None] * world
        dist.all_gather_object(parts, strip.u)
        if rank == 0:
            ref = u0
            for _ in range(3):
                ref = g.step(ref, dt)
            full = torch.cat(parts, 0)
            out.put(float((full - ref).abs().max() / ref.abs().max()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", ["periodic", "wall"])
def test_strip_exchange_equals_single_domain(case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_strip_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    err = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert err <= 1e-15, err


def _stats_worker(rank, world, port, out):
    _init(rank, world, port)
    try:
        x = torch.from_numpy(inputs.uniform_values(1000, seed=3, lo=0.0, hi=5.0) ** 2)
        lo, n = strip_rows(1000, world, rank)
        mine = x[lo:lo + n]
        m = mine.mean().item()
        sd = mine.std(unbiased=False).item()
        cnt, mean, m2 = gather_stats(n, m, sd)
        t = torch.tensor([float(rank + 1) * 1.5], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            out.put((cnt, mean, (m2 / cnt) ** 0.5, x.mean().item(), x.std(unbiased=False).item(), t.item()))
    finally:
        dist.destroy_process_group()


def test_chan_combination_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_stats_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    cnt, mean, std, gm, gs, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert cnt == 1000
    assert abs(mean - gm) <= 1e-13 * gm and abs(std - gs) <= 1e-12 * gs
    assert tmax == 3.0


def test_strip_rows_and_combine_stats_serial():
    assert [strip_rows(10, 3, r) for r in range(3)] == [(0, 4), (4, 3), (7, 3)]
    a = [1.0, 2.0, 4.0, 8.0, 16.0]
    t1 = (2, 1.5, 0.5)            # [1, 2]
    t2 = (3, 28.0 / 3, sum((v - 28.0 / 3) ** 2 for v in a[2:]))
    n, mean, m2 = combine_stats([t1, t2])
    ref = sum(a) / 5
    assert n == 5 and abs(mean - ref) < 1e-14 and abs(m2 - sum((v - ref) ** 2 for v in a)) < 1e-12
