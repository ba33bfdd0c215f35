"""Domain decomposition of a lattice into z-slabs, one per rank, with ghost planes.

Rank r of W owns the planes [z0, z1) of the global nz (near-equal split) and steps an
extended slab of nzl = (z1 - z0) + 2H planes: H ghost planes below and above its own.  The
step is the unmodified single-lattice step on the extended slab; its z-wrap joins the top
and bottom ghosts, so the ghost planes come out wrong, and after every step the ranks
exchange them: each rank's first H owned planes become its lower neighbour's top ghosts,
its last H owned planes its upper neighbour's bottom ghosts (periodic in rank).

Why H planes make every owned plane exact.  A node's state at t + 1 is pushed from the
collisions at its own plane and the planes next to it, and a collision reads the stencil
fields (densities, colour, psi) of the planes next to it: the new state of a plane depends
on the old state of the planes within 2 of it.  With the CG repulsion force the collision
also reads the interface normals of the neighbour planes, which are gradients of the
colour field: 3.  So with H = 2 (3 with the repulsion force) ghost planes that are exact
at t, every owned plane is exact at t + 1, and because every node is computed by the same
code from the same inputs, a decomposed run gives the single-domain result bit for bit.
The multirange SC model reaches two nodes: its collision reads fields at distance 2,
hence H = 3 as well.

Exchange volume.  Each step moves H planes of raw state (all K*Q populations and the K
reference densities) per face; the minimal exchange is the 5 populations per colour that
cross a face plus a density halo of 1 (2 with the repulsion force).  The ghost-plane form
trades that volume (and 2H redundant planes of work per rank) for running the tuned
single-lattice kernels unmodified.

Transports.  `dist_exchange` sends and receives the packed planes with torch.distributed
point-to-point operations (NCCL between GPUs, each message landing in the receiver's own
memory; gloo on CPU); `local_exchange` moves them between sub-domains held by one process.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np


def slab_bounds(nz: int, world: int, rank: int):
    """Planes [z0, z1) owned by `rank` of `world` (near-equal split)."""
    return (rank * nz) // world, ((rank + 1) * nz) // world


def ghost_planes(model: int, rep_pi: float = 0.0) -> int:
    """H: how far (in planes) one step's dependencies reach: 2, or 3 with the CG repulsion
    force or the multirange SC model (model 3)."""
    return 3 if (rep_pi != 0.0 and model == 0) or model == 3 else 2


@dataclass
class Slab:
    nz: int       # global planes
    world: int
    rank: int
    halo: int     # H
    z0: int = 0   # owned planes [z0, z1)
    z1: int = 0

    def __post_init__(self):
        self.z0, self.z1 = slab_bounds(self.nz, self.world, self.rank)
        if self.z1 - self.z0 < self.halo:
            raise ValueError(f"slab of {self.z1 - self.z0} planes is thinner than the {self.halo} ghost planes")

    @property
    def nzl(self) -> int:
        return self.z1 - self.z0 + 2 * self.halo

    def planes(self) -> np.ndarray:
        """Global plane index of every local plane (periodic)."""
        return (np.arange(self.z0 - self.halo, self.z1 + self.halo)) % self.nz

    def cut(self, field, plane_size: int):
        """The extended slab of a node-ordered field ([..., N] with N = nz * plane_size)."""
        if field is None:
            return None
        a = np.asarray(field)
        lead = a.shape[:-1]
        a = a.reshape(lead + (self.nz, plane_size))[..., self.planes(), :]
        return np.ascontiguousarray(a.reshape(lead + (self.nzl * plane_size,)))

    def owned(self, local_field, plane_size: int):
        """The owned planes of a local node-ordered field."""
        a = np.asarray(local_field)
        lead = a.shape[:-1]
        a = a.reshape(lead + (self.nzl, plane_size))[..., self.halo:self.halo + self.z1 - self.z0, :]
        return a.reshape(lead + ((self.z1 - self.z0) * plane_size,))


class SlabDomain:
    """One rank's sub-domain: an engine stepping the extended slab, and the ghost exchange.

    The engine provides step(n), get_planes(z0, n) -> packed planes and
    set_planes(z0, n, packed); `LatticeEngine` wraps a CUDA lattice (lbm.Lattice)."""

    def __init__(self, engine, slab: Slab):
        self.engine = engine
        self.slab = slab

    def outgoing(self):
        """(planes for the lower neighbour's top ghosts, planes for the upper neighbour's
        bottom ghosts): the first and the last H owned planes."""
        H, nzl = self.slab.halo, self.slab.nzl
        return self.engine.get_planes(H, H), self.engine.get_planes(nzl - 2 * H, H)

    def incoming(self, from_upper, from_lower):
        """Ghost planes received: the upper neighbour's first owned planes become the top
        ghosts, the lower neighbour's last owned planes the bottom ghosts."""
        H, nzl = self.slab.halo, self.slab.nzl
        self.engine.set_planes(nzl - H, H, from_upper)
        self.engine.set_planes(0, H, from_lower)


def local_exchange(domains):
    """Ghost exchange between the sub-domains of all ranks held by this process (rank
    order): rank r's top ghosts from rank r+1, its bottom ghosts from rank r-1 (periodic).
    All outgoing planes are read before any ghost is written."""
    out = [d.outgoing() for d in domains]
    w = len(domains)
    for r, d in enumerate(domains):
        d.incoming(out[(r + 1) % w][0], out[(r - 1) % w][1])


def dist_exchange(domain: SlabDomain, group=None):
    """Ghost exchange of this rank's sub-domain with its two z-neighbours over
    torch.distributed point-to-point messages (one world: the rank's own planes)."""
    import torch.distributed as dist
    world, rank = domain.slab.world, domain.slab.rank
    down, up = domain.outgoing()
    if world == 1:
        domain.incoming(down, up)
        return
    lower, upper = (rank - 1) % world, (rank + 1) % world
    from_upper, from_lower = down.clone(), up.clone()  # receive buffers of the same size
    ops = [dist.P2POp(dist.isend, down, lower, group), dist.P2POp(dist.isend, up, upper, group),
           dist.P2POp(dist.irecv, from_upper, upper, group), dist.P2POp(dist.irecv, from_lower, lower, group)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    domain.incoming(from_upper, from_lower)


class LatticeEngine:
    """A CUDA lattice (lbm.Lattice) stepping an extended slab; planes move as packed raw
    state (lbm_get_state_planes / lbm_set_state_planes) on the lattice's stream."""

    def __init__(self, lattice):
        self.lat = lattice

    def step(self, n: int = 1):
        self.lat.step(n)

    def get_planes(self, z0: int, n: int):
        buf = self.lat.state_planes(z0, n)
        self.lat.stream.synchronize()  # the buffer is read by another stream or process
        return buf

    def set_planes(self, z0: int, n: int, buf):
        self.lat.set_state_planes(z0, n, buf)


def lattice_slab(params, slab: Slab, rho_r, rho_b=None, u=None, solid=None, stream=None):
    """The CUDA lattice of `slab` (params of the global lattice), initialised from the
    global host fields, with its ghost planes made exact by one exchange (the caller runs
    it: local_exchange or dist_exchange)."""
    import torch
    from . import lbm
    p = replace(params, nz=slab.nzl)
    lat = lbm.Lattice(p, stream=stream)
    plane = params.nx * params.ny
    dev = lat.device
    t = lambda a, dt=torch.float64: None if a is None else torch.as_tensor(slab.cut(a, plane), dtype=dt, device=dev)
    lat.init(t(rho_r), t(rho_b), t(u), t(solid, torch.uint8))
    return SlabDomain(LatticeEngine(lat), slab)
