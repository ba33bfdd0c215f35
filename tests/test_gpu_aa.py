"""In-place (AA-pattern) streaming, LBM_STREAM_AA: the same step as the two-buffer scheme
with one population buffer, checked against the FP64 oracle after an even and an odd
number of steps (the two storage layouts), against the two-buffer path, through a
checkpoint taken at odd parity, and for the blow-up freeze.

Tolerances are those of test_gpu_parity.py: FP64 every population <= 1e-12 relative
(floor 1e-3 rho_max) after 100 and 101 steps; FP32 densities <= 1e-5 relative at every
node and velocities <= 1e-5 in L2 (the repulsion-force cases after 2 steps, see there);
FP16 storage within F16_TOL."""
import numpy as np
import pytest

from tests import cases as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts only to be deselected
    pytest.skip("needs a CUDA device", allow_module_level=True)


def _rho_max(case):
    return max(np.max(case.rho_r), 0.0 if case.rho_b is None else np.max(case.rho_b))


def _pops_rel_err(g, o, rho_max, floor=1e-3):
    return np.max(np.abs(g - o) / np.maximum(np.abs(o), floor * rho_max))


@pytest.mark.parametrize("name", list(C.SMALL_CASES))
def test_aa_fp64_parity_even_and_odd(orc, lbm, name):
    case = C.SMALL_CASES[name]()
    s = C.oracle_sim(orc, case)
    lat = C.gpu_lattice(lbm, case, lbm.FP64, streaming=lbm.STREAM_AA)
    rm = _rho_max(case)
    for steps in (100, 1):
        s.step(steps)
        lat.step(steps)
        err = _pops_rel_err(lat.pops().cpu().numpy(), s.pops(), rm)
        print(f"{name}: in-place FP64, +{steps} steps: max rel err {err:.2e}")
        assert err < 1e-12
    _, _, _, tot, rc = lat.moments()
    _, _, _, ot = s.moments()
    assert rc == lbm.OK
    for k, name_t in enumerate(lbm.TOTAL_NAMES):
        assert abs(tot[name_t] - ot[k]) <= 1e-11 * max(1.0, abs(ot[k])), name_t


@pytest.mark.parametrize("name", ["cg_drop3d", "cg_drop2d", "cg_walls3d", "sc_mp3d", "sc_2c3d", "sc_walls2d",
                                  "cg_rep3d", "cg_tma3d"])
def test_aa_fp32_parity(orc, lbm, name):
    case = C.SMALL_CASES[name]()
    rep = bool(case.kw.get("rep_pi"))
    steps = 2 if rep else 101
    s = C.oracle_sim(orc, case).step(steps)
    lat = C.gpu_lattice(lbm, case, lbm.FP32, streaming=lbm.STREAM_AA)
    t0, _ = lat.totals()
    lat.step(steps)
    rr, rb, u, tot, rc = lat.moments(device=False)
    orr, orb, ou, _ = s.moments()
    assert rc == lbm.OK
    scale = max(orr.max(), orb.max())
    fl = np.ones(orr.size, bool) if case.solid is None else case.solid == 0
    er = np.max((np.abs(rr - orr) / np.maximum(np.abs(orr), 1e-3 * scale))[fl])
    eb = np.max((np.abs(rb - orb) / np.maximum(np.abs(orb), 1e-3 * scale))[fl])
    eu2 = np.linalg.norm(u - ou) / np.linalg.norm(ou)
    print(f"{name}: in-place FP32 after {steps} steps: rho err {er:.2e}/{eb:.2e}, u err L2 {eu2:.2e}")
    assert er < 1e-5 and eb < 1e-5
    if rep:
        assert np.quantile(np.abs(u - ou).max(0), 0.99) / np.max(np.abs(ou)) < 3e-5
    else:
        assert eu2 < 1e-5
    for m in ("mass_r", "mass_b"):
        if t0[m] > 0:
            assert abs(tot[m] - t0[m]) <= 1e-6 * t0[m]


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("name", ["cg_drop3d", "sc_mp3d"])
def test_aa_16bit_storage(orc, lbm, name, precision):
    from tests.test_gpu_parity import F16_TOL
    case = C.SMALL_CASES[name]()
    s = C.oracle_sim(orc, case).step(100)
    lat = C.gpu_lattice(lbm, case, precision, streaming=lbm.STREAM_AA)
    t0, _ = lat.totals()
    lat.step(100)
    rr, rb, u, tot, rc = lat.moments(device=False)
    orr, orb, ou, _ = s.moments()
    assert rc == lbm.OK
    scale = max(orr.max(), orb.max())
    er = max(np.max(np.abs(rr - orr)), np.max(np.abs(rb - orb))) / scale
    eu = np.linalg.norm(u - ou) / np.linalg.norm(ou)
    dm = abs(tot["mass_r"] - t0["mass_r"]) / t0["mass_r"]
    print(f"{name} in-place precision {precision}: rho err {er:.2e}, u err {eu:.2e}, mass drift {dm:.2e}")
    tr, tu, tm = F16_TOL[precision]
    assert er < tr and eu < tu and dm < tm


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["cg_walls3d", "sc_2c3d"])
def test_aa_checkpoint_at_odd_parity(lbm, name, precision):
    """A state saved after an odd number of steps is written in the two-buffer layout: it
    resumes bitwise in a fresh in-place context, and loads into a two-buffer context
    (results there agree to rounding)."""
    case = C.SMALL_CASES[name]()
    solid = None if case.solid is None else torch.as_tensor(case.solid, dtype=torch.uint8, device="cuda")
    a = C.gpu_lattice(lbm, case, precision, streaming=lbm.STREAM_AA).step(41)
    raw = a.save_state()
    b = lbm.Lattice(lbm.Params(precision=precision, streaming=lbm.STREAM_AA, **case.kw)).load_state(raw, solid)
    ab = lbm.Lattice(lbm.Params(precision=precision, **case.kw)).load_state(raw, solid)
    ref = C.gpu_lattice(lbm, case, precision).step(41)
    # the saved state is the two-buffer state of the same step, to rounding
    pa, pr = b.pops().cpu().numpy(), ref.pops().cpu().numpy()
    scale = np.max(np.abs(pr))
    assert np.max(np.abs(pa - pr)) <= (1e-13 if precision == 0 else 1e-6) * scale
    for lat in (a, b, ab):
        lat.step(59)
    pa, pb, pab = (x.pops().cpu().numpy() for x in (a, b, ab))
    assert np.array_equal(pa, pb)
    assert np.max(np.abs(pab - pa)) <= (1e-12 if precision == 0 else 1e-5) * scale


def test_aa_blowup_freezes_the_state(lbm):
    case = C.cg_drop3d()
    rr = case.rho_r.copy()
    rr[5] = np.nan
    lat = lbm.Lattice(lbm.Params(precision=lbm.FP32, diag_every=1, streaming=lbm.STREAM_AA, **case.kw))
    lat.init(torch.as_tensor(rr, device=lat.device), torch.as_tensor(case.rho_b, device=lat.device))
    lat.step(3)
    p1 = lat.pops().cpu().numpy()
    lat.step(4)
    assert np.array_equal(lat.pops().cpu().numpy(), p1, equal_nan=True)
    tot, rc = lat.totals()
    assert rc == lbm.EUNSTABLE and tot["nonfinite"] > 0


def test_aa_full_size_matches_two_buffer(lbm):
    """128^3 droplet (the benchmark workload), 3 FP32 steps: in-place against the
    two-buffer cluster kernel, every population within a few ulps of the largest."""
    import bench
    rr, rb, _ = bench.workload_fields()
    t = lambda x: torch.as_tensor(x, dtype=torch.float64, device="cuda")
    out = []
    for streaming in (lbm.STREAM_AB, lbm.STREAM_AA):
        lat = lbm.Lattice(lbm.Params(precision=lbm.FP32, streaming=streaming, **bench.cg_kw()))
        lat.init(t(rr), t(rb))
        lat.step(3)
        out.append(lat.pops())
        assert lat.totals()[1] == lbm.OK
    d = (out[0] - out[1]).abs().max().item() / out[0].abs().max().item()
    print(f"128^3 CG FP32, 3 steps: in-place vs two-buffer max diff {d:.2e} of max|f|")
    assert d < 1e-6


def test_aa_not_accepted_by_batch(lbm):
    case = C.cg_drop3d()
    lat = C.gpu_lattice(lbm, case, lbm.FP32, streaming=lbm.STREAM_AA)
    b = lbm.Batch(lbm.FP32, 4, 64)
    with pytest.raises(lbm.LbmError):
        b.set([lat], [10])
