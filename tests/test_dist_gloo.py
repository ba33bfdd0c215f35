"""Multi-rank logic of bench.py on CPU: world size 2 over gloo (no GPU).  Each rank runs
independent replicas; the job's time is the slowest rank's (all-reduce MAX) and the
whole-job throughput counts every rank's lattice updates."""
import os
import socket

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
    with mp.Manager() as m:
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
