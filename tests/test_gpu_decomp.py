"""z-slab domain decomposition (decomp.py) on one GPU: two or three sub-domains of a lattice,
each an extended slab stepped by the library's own kernels, their ghost planes moved with
lbm_get_state_planes / lbm_set_state_planes (device copies); after every step the owned
planes equal the single-domain run's raw state bit for bit.  (The kernels compute every
node with the same code from the same inputs whatever the lattice's nz, so the result
does not depend on the partition.)  Several GPUs would move the same planes with NCCL
point-to-point messages (decomp.dist_exchange, tested over gloo on CPU); this pool gives
one GPU per run, so the multi-GPU path is not measured on hardware."""
import numpy as np
import pytest

import tests.cases as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


CASES = {
    "cg_fp32_cluster": (lambda: C.cg_drop3d(nx=64, ny=32, nz=40), 1, (64, 4, 0)),   # cluster TMA kernel
    "sc_fp32_ring": (lambda: C.sc_mp3d(nx=64, ny=16, nz=36), 1, (64, 4, 0)),       # ring kernel
    "cg_fp16_ring": (lambda: C.cg_drop3d(nx=64, ny=32, nz=30), 2, (32, 16, 0)),    # ring kernel, 16-bit
    "cg_rep_fp64": (C.cg_rep3d, 0, (32, 8, 16)),                                   # repulsion, H = 3
    "cg_walls_fp32": (C.cg_walls3d, 1, (32, 8, 16)),                               # walls, body force
    "sc_mr_fp32": (lambda: C.sc_mr3d(nx=20, ny=16, nz=24), 1, (32, 8, 0)),          # multirange, H = 3
    "sc_mr_walls_fp64": (lambda: C.sc_mr3d(nz=18, walls=True), 0, (32, 8, 0)),      # multirange with walls
}


@pytest.mark.parametrize("name,world", [(n, 2) for n in CASES] + [("cg_fp32_cluster", 3), ("sc_mr_fp32", 3)])
def test_slabs_on_one_gpu_match_single_domain(lbm, name, world):
    from paper_2110_05197_gb300 import decomp
    make, precision, tiling = CASES[name]
    case = make()
    kw = case.kw
    params = lbm.Params(precision=precision, **kw)
    steps = 25
    full = C.gpu_lattice(lbm, case, precision)
    full.set_tiling(*tiling)
    full.step(steps)
    H = decomp.ghost_planes(kw["model"], kw.get("rep_pi", 0.0))
    doms = [decomp.lattice_slab(params, decomp.Slab(kw["nz"], world, r, H), case.rho_r, case.rho_b, case.u,
                                case.solid) for r in range(world)]
    for d in doms:
        d.engine.lat.set_tiling(*tiling)
    decomp.local_exchange(doms)
    for _ in range(steps):
        for d in doms:
            d.engine.step(1)
        decomp.local_exchange(doms)
    torch.cuda.synchronize()
    nb_plane = full.state_planes(0, 1).numel()
    for d in doms:
        s = d.slab
        got = d.engine.lat.state_planes(s.halo, s.z1 - s.z0).cpu().numpy()
        want = full.state_planes(s.z0, s.z1 - s.z0).cpu().numpy()
        assert got.size == want.size == nb_plane * (s.z1 - s.z0)
        assert np.array_equal(got, want), (name, s.rank)
    print(f"{name}: {world} slabs of {[d.slab.z1 - d.slab.z0 for d in doms]} planes (+{2 * H} ghosts) "
          f"== single domain after {steps} steps")
