"""The multicomponent Shan-Chen model with multirange potentials (Eq. benziforces) on the
GPU's field-pass kernels, beyond the small parity cases of test_gpu_parity.py and
test_gpu_aa.py (which include it): 16-bit storage against the oracle, a 48^3 droplet
against the oracle every population, and the in-place mode against two buffers."""
import numpy as np
import pytest

from paper_2110_05197_gb300 import inputs
from tests import cases as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts only to be deselected
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.mark.parametrize("precision", [2, 3])
def test_multirange_16bit_storage(orc, lbm, precision):
    from tests.test_gpu_parity import F16_TOL
    case = C.sc_mr3d()
    s = C.oracle_sim(orc, case).step(100)
    lat = C.gpu_lattice(lbm, case, precision)
    t0, _ = lat.totals()
    lat.step(100)
    rr, rb, u, tot, rc = lat.moments(device=False)
    orr, orb, ou, _ = s.moments()
    assert rc == lbm.OK
    scale = max(orr.max(), orb.max())
    er = max(np.max(np.abs(rr - orr)), np.max(np.abs(rb - orb))) / scale
    eu = np.linalg.norm(u - ou) / np.linalg.norm(ou)
    dm = abs(tot["mass_r"] - t0["mass_r"]) / t0["mass_r"]
    print(f"multirange precision {precision}: rho err {er:.2e}, u err {eu:.2e}, mass drift {dm:.2e}")
    tr, tu, tm = F16_TOL[precision]
    assert er < tr and eu < tu and dm < tm


def _drop48():
    n = 48
    ins = inputs.sphere(n, n, n, 10.0)
    rr = np.where(ins, 1.18, 0.18) * (1 + 0.01 * inputs.uniform_pm1(9, n ** 3, 0))
    rb = np.where(ins, 0.18, 1.18) * (1 + 0.01 * inputs.uniform_pm1(9, n ** 3, 1))
    kw = dict(lattice=1, model=3, nx=n, ny=n, nz=n, Ga=(-9.0, -8.0), Gr=(8.1, 7.1), G=1.215, rho0_psi=0.83)
    return C.Case("mr_drop48", kw, rr, rb)


@pytest.mark.parametrize("streaming", [0, 1])
def test_multirange_48cube_fp32_every_population(orc, lbm, streaming):
    case = _drop48()
    s = C.oracle_sim(orc, case).step(3)
    lat = C.gpu_lattice(lbm, case, lbm.FP32, streaming=streaming).step(3)
    g, o = lat.pops().cpu().numpy(), s.pops()
    err = np.max(np.abs(g - o)) / np.max(np.abs(o))
    print(f"multirange 48^3 FP32 streaming {streaming}, 3 steps: max |err| / max|f| {err:.2e}")
    assert err < 1e-6


def test_multirange_inplace_matches_two_buffer(lbm):
    case = C.sc_mr3d()
    a = C.gpu_lattice(lbm, case, lbm.FP64).step(37)
    b = C.gpu_lattice(lbm, case, lbm.FP64, streaming=lbm.STREAM_AA).step(37)
    pa, pb = a.pops().cpu().numpy(), b.pops().cpu().numpy()
    assert np.max(np.abs(pa - pb)) <= 1e-13 * np.max(np.abs(pa))
