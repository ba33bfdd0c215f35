"""lbm_totals_noalloc: the allocation-free entry point for callers that cannot call
cudaMalloc (its scratch is a static device array).  Checked through the C ABI against the
totals of the existing entry point (lbm_moments) on two calls in a row, to the same
rounding tolerance as the other FP64 reductions.  Kept in a file pytest collects last."""
import numpy as np
import pytest

from tests import cases as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def lbm():
    from paper_2110_05197_gb300 import build, lbm as L
    build.build()
    return L


def _close(a, b):
    scale = max(1.0, float(np.max(np.abs(b[:2]))))
    for k in range(len(b)):
        tol = 1e-12 * max(abs(b[k]), 1.0 if k in (0, 1, 8, 9) else 0.0) + 1e-13 * (scale if k < 5 else 1.0)
        assert abs(a[k] - b[k]) <= tol, (k, a[k], b[k])


@pytest.mark.parametrize("name,precision", [("cg_walls3d", 1), ("sc_mp3d", 0), ("sc_2c3d", 1), ("cg_drop2d", 0)])
def test_noalloc_totals_match_moments_twice(lbm, name, precision):
    case = C.SMALL_CASES[name]()
    lat = C.gpu_lattice(lbm, case, precision).step(30)
    want, rc = lat.totals()
    want = np.array([want[k] for k in lbm.TOTAL_NAMES])
    pops = lat.pops()
    solid = None if case.solid is None else torch.as_tensor(case.solid, dtype=torch.uint8, device=lat.device)
    # first call writes a device buffer, the second a host one
    dev_out = torch.zeros(lbm.NTOTALS, dtype=torch.float64, device=lat.device)
    _, rc1 = lbm.totals_noalloc(lat.params, pops, solid, dev_out, lat.stream)
    got1 = dev_out.cpu().numpy()
    got2, rc2 = lbm.totals_noalloc(lat.params, pops, solid, None, lat.stream)
    assert rc1 == lbm.OK and rc2 == lbm.OK
    _close(got1, want)
    _close(got2, want)


def test_noalloc_rejects_sizes_beyond_its_scratch(lbm):
    p = lbm.Params(nx=102, ny=102, nz=102)  # 1,061,208 nodes > LBM_NOALLOC_MAX_NODES
    assert p.n > lbm.NOALLOC_MAX_NODES
    pops = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.totals_noalloc(p, pops)
    assert e.value.status == lbm.EINVAL
