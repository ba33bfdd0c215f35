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


def _raw_call(lbm, params, pops, solid=None):
    """The C entry point itself, without the binding's argument checks."""
    import ctypes
    out = np.zeros(lbm.NTOTALS)
    cp = params.to_c()
    return lbm.lib().lbm_totals_noalloc(ctypes.byref(cp), pops.data_ptr(),
                                        None if solid is None else solid.data_ptr(), out.ctypes.data,
                                        torch.cuda.current_stream().cuda_stream)


def test_noalloc_rejects_sizes_beyond_its_scratch(lbm):
    p = lbm.Params(nx=102, ny=102, nz=102)  # 1,061,208 nodes > LBM_NOALLOC_MAX_NODES
    assert p.n > lbm.NOALLOC_MAX_NODES
    pops = torch.zeros(16, dtype=torch.float64, device="cuda")
    # the C side refuses the size before it reads anything
    assert _raw_call(lbm, p, pops) == lbm.EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm.totals_noalloc(p, pops)
    assert e.value.status == lbm.EINVAL


def test_noalloc_rejects_the_repulsion_force(lbm):
    """CG with the repulsion force: the force enters u and E_kin, which this entry point
    does not compute, so the state is refused instead of given other totals."""
    case = C.cg_rep3d()
    lat = C.gpu_lattice(lbm, case, lbm.FP64)
    assert _raw_call(lbm, lat.params, lat.pops()) == lbm.EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm.totals_noalloc(lat.params, lat.pops())
    assert e.value.status == lbm.EINVAL


def test_noalloc_rejects_bad_buffers(lbm):
    case = C.sc_2c3d()
    lat = C.gpu_lattice(lbm, case, lbm.FP64).step(2)
    p, pops = lat.params, lat.pops()
    # host memory is not device memory: the C side refuses it
    assert _raw_call(lbm, p, pops.cpu().pin_memory()) == lbm.EINVAL
    bad = [
        (pops.float(), None),                                 # wrong dtype
        (pops[:-1], None),                                    # too small
        (pops.view(2, -1).t().contiguous().t(), None),        # not contiguous
        (pops, torch.zeros(p.n, dtype=torch.float32, device=pops.device)),  # solid not uint8
        (pops, torch.zeros(p.n - 1, dtype=torch.uint8, device=pops.device)),  # solid too small
        (pops.cpu(), None),                                   # not a CUDA tensor
    ]
    for pp, solid in bad:
        with pytest.raises(lbm.LbmError) as e:
            lbm.totals_noalloc(p, pp, solid)
        assert e.value.status == lbm.EINVAL
    # the state itself is still accepted
    _, rc = lbm.totals_noalloc(p, pops)
    assert rc == lbm.OK
