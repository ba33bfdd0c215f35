"""Lattices whose population index K * Q * N passes 2^31 run the step kernels with 64-bit
indices, all smaller ones with 32-bit indices.  No oracle reaches that size, so the test
uses periodicity: a 384^3 colour-gradient lattice (38 * 384^3 = 2,151,677,952 > 2^31)
initialised with a 48^3 state tiled 8 x 8 x 8 keeps that period, and since every node is
computed by the same per-node code, its densities and velocities after a few steps equal
the 48^3 lattice's (32-bit path), tiled, bit for bit.  Both lattices use the generic
plane-marching kernel (16 x 8 tiles), then in-place streaming (field-pass kernels).  The
batched launch, which indexes in 32 bits, refuses the large lattice."""
import numpy as np
import pytest

from tests import cases as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

SMALL, REPS = 48, 8
BIG = SMALL * REPS


@pytest.fixture(scope="module")
def lbm():
    from paper_2110_05197_gb300 import build, lbm as L
    build.build()
    return L


def _tile(a):
    return np.tile(a.reshape(SMALL, SMALL, SMALL), (REPS, REPS, REPS)).ravel()


def _moments(lat):
    rr, rb, u, _, rc = lat.moments()
    return rr.cpu().numpy(), rb.cpu().numpy(), u.cpu().numpy(), rc


@pytest.mark.parametrize("streaming", ["ab", "aa"])
def test_64bit_index_path_matches_the_tiled_small_lattice(lbm, streaming):
    free, _ = torch.cuda.mem_get_info()
    if free < 40 * 2 ** 30:
        pytest.skip("needs about 25 GB of free device memory")
    assert 38 * BIG ** 3 >= 2 ** 31 > 38 * SMALL ** 3
    case = C.cg_drop3d(nx=SMALL, ny=SMALL, nz=SMALL, seed=7)
    mode = lbm.STREAM_AA if streaming == "aa" else lbm.STREAM_AB
    steps = 3  # in place: even, odd and even layout parity
    small = C.gpu_lattice(lbm, case, lbm.FP32, streaming=mode)
    small.set_tiling(16, 8, 0)
    small.step(steps)
    srr, srb, su, rc = _moments(small)
    assert rc == lbm.OK
    small.close()

    kw = dict(case.kw, nx=BIG, ny=BIG, nz=BIG)
    big = lbm.Lattice(lbm.Params(precision=lbm.FP32, streaming=mode, **kw))
    dev = big.device
    big.init(torch.as_tensor(_tile(case.rho_r), device=dev), torch.as_tensor(_tile(case.rho_b), device=dev))
    big.set_tiling(16, 8, 0)
    if streaming == "ab":
        # the batched kernel indexes in 32 bits: the large lattice is refused
        batch = lbm.Batch(lbm.FP32, 1, lbm.Batch.units(big), stream=big.stream)
        with pytest.raises(lbm.LbmError) as e:
            batch.set([big], [1])
        assert e.value.status == lbm.EINVAL
    big.step(steps)
    brr, brb, bu, rc = _moments(big)
    assert rc == lbm.OK
    big.close()
    assert np.array_equal(brr, _tile(srr))
    assert np.array_equal(brb, _tile(srb))
    assert np.array_equal(bu.reshape(3, -1), np.stack([_tile(c) for c in su.reshape(3, -1)]))
