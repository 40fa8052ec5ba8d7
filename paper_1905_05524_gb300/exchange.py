"""Strip decomposition of a uniform mesh across ranks.

ADER-DG exchanges data once per step (Sec. 1 of the paper: the scheme is
communication avoiding): after the element-local predictor, only the face
traces along partition edges are needed by the neighbour.  Here the mesh is
cut into horizontal strips of rows, one per rank; a step is

    predictor -> send edge traces to the ranks below/above -> install the
    received traces as halos -> corrector,

and the refinement statistics are combined across ranks with Chan et al.'s
pairwise update in rank order.  The stepping is backend-agnostic: a backend
provides predictor(dt), boundary_traces() -> (south, north) tensors,
set_halo(south, north) and corrector(dt).  `LibraryStrip` is the GPU backend
(libaderdg.so with bc_y = ADG_BC_EXCHANGE*); the tests drive the same
exchange with CPU ranks over gloo.
"""
import ctypes

import torch
import torch.distributed as dist

from . import _lib as L
from .solver import Mesh, _stream_ptr

TAG_UP, TAG_DOWN = 0, 1


def strip_rows(ny, world, rank):
    """(first row, number of rows) of `rank`'s strip of ny rows."""
    base, rem = divmod(ny, world)
    rows = base + (1 if rank < rem else 0)
    first = rank * base + min(rank, rem)
    return first, rows


def strip_bc(rank, world, periodic):
    """bc_y of a strip: periodic domains exchange on both sides; walled ones
    keep the wall on the outer strips."""
    if periodic:
        return L.ADG_BC_EXCHANGE
    if world == 1:
        return L.ADG_BC_WALL
    if rank == 0:
        return L.ADG_BC_WALL_EXCHANGE
    if rank == world - 1:
        return L.ADG_BC_EXCHANGE_WALL
    return L.ADG_BC_EXCHANGE


def neighbours(rank, world, periodic):
    below = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    above = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return below, above


def exchange_halos(south, north, rank, world, periodic, group=None):
    """Send this strip's edge traces to its neighbours and receive theirs.

    Returns (south_halo, north_halo): the north traces of the strip below and
    the south traces of the strip above (None where a wall closes the side)."""
    below, above = neighbours(rank, world, periodic)
    if world == 1:
        return (north.clone(), south.clone()) if periodic else (None, None)
    south_halo = torch.empty_like(south) if below is not None else None
    north_halo = torch.empty_like(north) if above is not None else None
    # sends (north up, south down) then receives (from below, from above): with
    # two ranks on a periodic domain both neighbours are the same rank, and
    # this order pairs the messages correctly also for backends that match
    # point-to-point messages by order rather than by tag
    ops = []
    if above is not None:
        ops.append(dist.P2POp(dist.isend, north, above, group, TAG_UP))
    if below is not None:
        ops.append(dist.P2POp(dist.isend, south, below, group, TAG_DOWN))
    if below is not None:
        ops.append(dist.P2POp(dist.irecv, south_halo, below, group, TAG_UP))
    if above is not None:
        ops.append(dist.P2POp(dist.irecv, north_halo, above, group, TAG_DOWN))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return south_halo, north_halo


class StripStepper:
    """One rank's strip: one face-trace exchange per step."""

    def __init__(self, backend, rank, world, periodic, group=None):
        self.b, self.rank, self.world, self.periodic, self.group = backend, rank, world, periodic, group

    def step(self, dt):
        self.b.predictor(dt)
        s, n = self.b.boundary_traces()
        hs, hn = exchange_halos(s, n, self.rank, self.world, self.periodic, self.group)
        self.b.set_halo(hs, hn)
        self.b.corrector(dt)


def combine_stats(triples):
    """Chan et al. pairwise combination of (count, mean, M2) triples, in the
    given (rank) order; returns (count, mean, M2)."""
    n, mean, m2 = triples[0]
    for nb, mb, m2b in triples[1:]:
        tot = n + nb
        d = mb - mean
        mean = mean + d * nb / tot
        m2 = m2 + m2b + d * d * n * nb / tot
        n = tot
    return n, mean, m2


def gather_stats(count, mean, std, group=None):
    """All ranks' (count, mean, M2) combined in rank order (CPU tensors)."""
    world = dist.get_world_size(group)
    local = torch.tensor([count, mean, std * std * count], dtype=torch.float64)
    allv = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allv, local, group=group)
    return combine_stats([tuple(float(x) for x in t) for t in allv])


class LibraryStrip:
    """GPU backend of StripStepper on libaderdg.so (bc_y = ADG_BC_EXCHANGE*)."""

    def __init__(self, mesh: Mesh):
        self.m = mesh
        n = mesh.cfg.degree + 1
        self.rec = mesh.cfg.nx * 17 * n
        self.south = torch.empty(self.rec, dtype=torch.float64, device=mesh.device)
        self.north = torch.empty_like(self.south)

    def predictor(self, dt):
        self.m.predictor(dt)

    def boundary_traces(self):
        L.check(self.m._lib.adg_get_boundary_traces(self.m.h, ctypes.c_void_p(self.south.data_ptr()),
                                                    ctypes.c_void_p(self.north.data_ptr()), _stream_ptr()))
        return self.south, self.north

    def set_halo(self, south, north):
        sp = ctypes.c_void_p(south.data_ptr()) if south is not None else None
        npn = ctypes.c_void_p(north.data_ptr()) if north is not None else None
        L.check(self.m._lib.adg_set_halo_traces(self.m.h, sp, npn, _stream_ptr()))

    def corrector(self, dt):
        self.m.corrector(dt)
