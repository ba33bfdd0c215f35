"""Batched stepping (lbm_batch_*) and the serving loop on the GPU.

* A lattice's result is bitwise the same alone and in a mix of other lattices (different
  grids, lattices, models, with and without walls), with jobs joining and finishing at
  different times, with and without CUDA-graph replay.
* Batched FP32 agrees with the oracle within the FP32 bounds of test_gpu_parity.
* The batch serving loop (FP16 storage) answers a small sweep with the same results as
  the plain FP32 one-at-a-time loop within the FP16 storage bounds.
"""
import numpy as np
import pytest

import tests.cases as C

pytestmark = pytest.mark.gpu


def _mix(lbm, precision):
    """Eight small lattices: D3Q19/D2Q9, CG/SC-MP/SC-2C, ragged sizes, two with walls."""
    cases = [C.cg_drop3d(nx=20, ny=18, nz=17), C.cg_drop3d(nx=37, ny=21, nz=19, ratio=4.0, seed=3),
             C.sc_mp3d(nx=24, ny=16, nz=20), C.sc_2c3d(nx=19, ny=23, nz=18), C.cg_drop2d(n=40),
             C.cg_drop2d(n=33, seed=4), C.cg_walls3d(), C.sc_walls2d()]
    return cases, [C.gpu_lattice(lbm, c, precision) for c in cases]


@pytest.mark.parametrize("precision", [1, 2])
def test_batch_alone_equals_mix(lbm, precision):
    import torch
    steps = [30, 17, 25, 30, 12, 22, 26, 19]
    cases, lats = _mix(lbm, precision)
    stream = lats[0].stream
    b = lbm.Batch(precision, 16, 4096, stream=stream)
    # jobs 0-3 and 6 start together; 4, 5 and 7 join after 8 steps (continuous batching)
    first = [0, 1, 2, 3, 6]
    b.set([lats[j] for j in first], [steps[j] for j in first])
    b.step(8, graph=True)
    b.set(lats, [max(0, steps[j] - 8) if j in first else steps[j] for j in range(len(lats))])
    for _ in range(4):
        b.step(7, graph=True)
    torch.cuda.synchronize()
    mixed = [lat.pops().cpu().numpy() for lat in lats]
    for j, case in enumerate(cases):
        for graph in (True, False):
            lat = C.gpu_lattice(lbm, case, precision)
            one = lbm.Batch(precision, 1, 4096, stream=lat.stream)
            one.set([lat], [steps[j]])
            for _ in range(-(-steps[j] // 5)):   # calls past the job's step count are no-ops for it
                one.step(5, graph=graph)
            torch.cuda.synchronize()
            assert np.array_equal(lat.pops().cpu().numpy(), mixed[j]), (case.name, graph)


def test_batch_fp32_matches_oracle(orc, lbm):
    import torch
    cases = [C.cg_drop3d(), C.sc_mp3d(), C.cg_drop2d(), C.cg_walls3d(), C.sc_walls2d()]
    lats = [C.gpu_lattice(lbm, c, lbm.FP32) for c in cases]
    b = lbm.Batch(lbm.FP32, 8, 4096, stream=lats[0].stream)
    b.set(lats, [100] * len(cases))
    b.step(100)
    torch.cuda.synchronize()
    for case, lat in zip(cases, lats):
        o = C.oracle_sim(orc, case)
        o.step(100)
        orr, orb, ou, _ = o.moments()
        rr, rb, u, tot, rc = lat.moments(device=False)
        assert rc == lbm.OK
        fl = np.ones(orr.size, bool) if case.solid is None else case.solid == 0
        er = np.max(np.abs(rr - orr)[fl]) / np.max(np.abs(orr))
        eu = np.linalg.norm(u - ou) / np.linalg.norm(ou)
        print(f"batched FP32 {case.name}: rho err {er:.2e}, u err L2 {eu:.2e}")
        assert er < 1e-5 and eu < 1e-5


def test_batch_rejects_unsupported_jobs(lbm):
    lat = C.gpu_lattice(lbm, C.cg_rep3d(), lbm.FP32)             # repulsion force
    b = lbm.Batch(lbm.FP32, 4, 1024, stream=lat.stream)
    with pytest.raises(lbm.LbmError):
        b.set([lat], [10])
    lat16 = C.gpu_lattice(lbm, C.cg_drop3d(), lbm.FP16)          # precision mismatch
    with pytest.raises(lbm.LbmError):
        b.set([lat16], [10])
    big = C.gpu_lattice(lbm, C.cg_drop3d(nx=64, ny=64, nz=64), lbm.FP32)
    with pytest.raises(lbm.LbmError):                            # table capacity
        lbm.Batch(lbm.FP32, 4, 8, stream=big.stream).set([big], [1])
    with pytest.raises(lbm.LbmError):
        lbm.Batch(lbm.FP64, 4, 8)


def test_serving_batch_matches_plain(lbm):
    from paper_2110_05197_gb300 import serve
    reqs = serve.sweep(10, seed=7, steps=(40, 120), rate_hz=200.0,
                       grids=[(64, 64, 1), (32, 32, 32), (24, 24, 24), (48, 32, 16)])
    plain = {r.rid: r for r in serve.PlainServer(lbm.FP32, keep_fields=True).run(reqs)}
    # 32^3 and 48 x 32 x 16 go to the large-lattice path (own kernel, second stream)
    batch = {r.rid: r for r in serve.BatchServer(lbm.FP16, budget_bytes=64 << 20, tick=16, batch_max_nodes=20_000,
                                                 keep_fields=True).run(reqs)}
    assert set(plain) == set(batch) == {r.rid for r in reqs}
    for r in reqs:
        a, b = plain[r.rid], batch[r.rid]
        if a.status != lbm.OK or b.status != lbm.OK:
            assert a.status == b.status, r
            continue
        err = np.max(np.abs(a.rho_r - b.rho_r)) / np.max(np.abs(a.rho_r))
        dm = abs(a.totals["mass_r"] - b.totals["mass_r"]) / a.totals["mass_r"]
        print(f"request {r.rid} {r.grid} model {r.model}: rho err {err:.2e}, mass {dm:.2e}")
        assert err < 5e-3 and dm < 1e-4
    s = serve.summary(list(batch.values()))
    assert s["p99_s"] >= s["p50_s"] > 0 and s["sims_per_hour"] > 0


def test_batch_chunk_length_does_not_change_results(lbm):
    """A job's z-chunk length in the batched launch (its tiling's tz, picked by the batch
    autotuner) changes only the work partition: the state is bitwise the same."""
    import torch
    from paper_2110_05197_gb300 import tune
    outs = []
    for tz in (4, 16, 0):
        cases, lats = _mix(lbm, lbm.FP16)
        for lat in lats[:4]:          # the 3-D lattices
            lat.set_tiling(32, 8, tz)
        b = lbm.Batch(lbm.FP16, 16, 4096, stream=lats[0].stream)
        b.set(lats, [20] * len(lats))
        b.step(20)
        torch.cuda.synchronize()
        outs.append([lat.pops().cpu().numpy() for lat in lats])
    for other in outs[1:]:
        for a, b_ in zip(outs[0], other):
            assert np.array_equal(a, b_)
    p = lbm.Params(lattice=lbm.D3Q19, model=lbm.CG, precision=lbm.FP16, nx=32, ny=32, nz=32, rho_b0=0.1)
    assert tune.batch_chunk(p) in tune.BATCH_CHUNKS
