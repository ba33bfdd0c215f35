"""Multi-rank logic on CPU: world size 2 over gloo (no GPU).

* bench.py: each rank runs independent replicas; the job's time is the slowest rank's
  (all-reduce MAX) and the whole-job throughput counts every rank's lattice updates.
* The z-slab domain decomposition (decomp.py) with ghost-plane exchange by point-to-point
  messages, each rank stepping its slab on the oracle: bitwise the single-domain run."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t = bench.slowest_rank(10.0 + 5.0 * rank)       # rank 1 is the slower replica
        v = bench.job_mlups(128 ** 3, 2, 50, world, t / 1e3)
        out[rank] = (t, v)
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_job_throughput_over_gloo():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for t, v in res.values():
        assert t == pytest.approx(15.0)                  # max over ranks
        assert v == pytest.approx(2 * 128 ** 3 * 50 * world / 15e-3 / 1e6)


def test_single_process_is_identity():
    import bench
    assert bench.slowest_rank(3.25) == 3.25
    assert bench.job_mlups(1000, 1, 10, 1, 1e-3) == pytest.approx(10.0)


# ---- z-slab domain decomposition (paper_2110_05197_gb300/decomp.py) on the oracle --------

class _OracleEngine:
    """The FP64 oracle stepping one extended slab (test infrastructure): planes move as
    float64 tensors of the canonical populations [K][Q][planes]."""

    def __init__(self, orc, params, rho_r, rho_b, u, solid):
        self.orc = orc
        self.p = params
        self.plane = params.nx * params.ny
        self.solid = solid
        self.sim = orc.OracleSim(params).init(rho_r, rho_b, u, solid)

    def step(self, n=1):
        self.sim.step(n)

    def get_planes(self, z0, n):
        import torch
        f = self.sim.pops()
        k, q, _ = f.shape
        f = f.reshape(k, q, self.p.nz, self.plane)[:, :, z0:z0 + n, :]
        return torch.from_numpy(np.ascontiguousarray(f).reshape(-1))

    def set_planes(self, z0, n, buf):
        f = self.sim.pops()
        k, q, _ = f.shape
        f = f.reshape(k, q, self.p.nz, self.plane)
        f[:, :, z0:z0 + n, :] = buf.numpy().reshape(k, q, n, self.plane)
        self.sim.init(np.zeros(self.p.n), None, None, self.solid, f.reshape(k, q, -1))


def _decomp_worker(rank, world, port, name, steps, out):
    import dataclasses
    import torch.distributed as dist
    import oracle
    from tests import cases as C
    from paper_2110_05197_gb300 import decomp
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        oracle.set_threads(2)
        case = _DECOMP_CASES[name]()
        kw = case.kw
        H = decomp.ghost_planes(kw["model"], kw.get("rep_pi", 0.0))
        slab = decomp.Slab(kw["nz"], world, rank, H)
        plane = kw["nx"] * kw["ny"]
        p = dataclasses.replace(oracle.Params(**kw), nz=slab.nzl)
        eng = _OracleEngine(oracle, p, slab.cut(case.rho_r, plane), slab.cut(case.rho_b, plane),
                            slab.cut(case.u, plane), slab.cut(case.solid, plane))
        dom = decomp.SlabDomain(eng, slab)
        decomp.dist_exchange(dom)   # make the ghosts exact (the init's gradients wrap in z)
        for _ in range(steps):
            eng.step(1)
            decomp.dist_exchange(dom)
        f = eng.sim.pops()
        out[rank] = (slab.z0, slab.z1, np.ascontiguousarray(slab.owned(f, plane)))
    finally:
        dist.destroy_process_group()


def _decomp_cases():
    from tests import cases as C
    return {
        "cg_drop3d": lambda: C.cg_drop3d(nx=20, ny=18, nz=16),
        "sc_mp3d": lambda: C.sc_mp3d(nx=16, ny=14, nz=12),
        "cg_walls3d": C.cg_walls3d,                       # walls in y, body force
        "cg_rep3d": C.cg_rep3d,                           # repulsion force: 3 ghost planes
    }


_DECOMP_CASES = _decomp_cases()


@pytest.mark.parametrize("name", list(_DECOMP_CASES))
def test_slab_decomposition_matches_single_domain_over_gloo(orc, name):
    """Two gloo ranks each step their z-slab (H ghost planes, exchanged every step by
    point-to-point messages) on the oracle; the assembled owned planes equal the
    single-domain oracle's populations bit for bit after 12 steps (Sec. 2.3: a layer of
    boundary nodes shared between processes suffices; here H = 2, 3 with the repulsion
    force)."""
    world, steps = 2, 12
    case = _DECOMP_CASES[name]()
    ref = orc.OracleSim(orc.Params(**case.kw)).init(case.rho_r, case.rho_b, case.u, case.solid).step(steps).pops()
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_decomp_worker, args=(world, port, name, steps, out), nprocs=world, join=True)
        res = dict(out)
    kw = case.kw
    plane = kw["nx"] * kw["ny"]
    k, q = ref.shape[:2]
    full = ref.reshape(k, q, kw["nz"], plane)
    for rank in range(world):
        z0, z1, owned = res[rank]
        mine = owned.reshape(k, q, z1 - z0, plane)
        assert np.array_equal(mine, full[:, :, z0:z1, :]), (name, rank)
