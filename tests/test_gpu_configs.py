"""GPU parity at the full sizes of the paper-scale workloads (the benchmark's 128^3
droplet is covered in test_gpu_parity.py):

* D2Q9 colour-gradient static droplet, 128 x 128, FP64, the whole 2000-step run (Laplace
  test of Sec. 3.1): every population against the oracle;
* Rayleigh-Plateau jet, 64 x 64 x 512 (Sec. 3.4), CG and two-component SC: two FP32 steps
  against the oracle, every population; FP16 and BF16 storage against FP32 over 50 steps;
* high-density-ratio ligament, 96 x 96 x 768, ratio 1000, viscosity ratio 50 (Sec. 3.3),
  both colour-field definitions: two FP64 steps against the oracle (the sharp-interface
  start at this ratio is too violent for FP32 cancellation, see the test);
* dense emulsion, 256^3, 200 droplets with the CG repulsion force (Sec. 3.6): two FP32 steps
  against the oracle (densities element-wise; the repulsion force's Heaviside decisions
  may flip at FP32 resolution, so u is checked on its 99% quantile).

The oracle runs the same inputs on the host cores (a few seconds per step at 256^3).
"""
import numpy as np
import pytest

import tests.cases as C
from paper_2110_05197_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _pop_err(g, o, rho_max, floor=1e-3):
    return np.max(np.abs(g - o) / np.maximum(np.abs(o), floor * rho_max))


def test_config1_static_droplet_2000_steps_fp64(orc, lbm):
    n = 128
    rr, rb = inputs.two_fluid(inputs.sphere(n, n, 1, 20.0), 1.0, 1.0, 0.0, 1)
    case = C.Case("droplet2d", dict(lattice=0, model=0, nx=n, ny=n, nz=1, rho_r0=1.0, rho_b0=1.0, A=1e-2), rr, rb)
    s = C.oracle_sim(orc, case)
    lat = C.gpu_lattice(lbm, case, lbm.FP64)
    s.step(100)
    lat.step(100)
    err100 = _pop_err(lat.pops().cpu().numpy(), s.pops(), 1.0)
    s.step(1900)
    lat.step(1900)
    err = _pop_err(lat.pops().cpu().numpy(), s.pops(), 1.0)
    print(f"D2Q9 128^2 FP64: max relative population error {err100:.2e} after 100 steps, {err:.2e} after 2000")
    # the stated FP64 bound holds at 100 steps; the two sides round differently (operation
    # order, fused multiply-adds), and the interface dynamics grow those differences, so
    # the whole run is held to ten times that bound
    assert err100 < 1e-12
    assert err < 1e-11


def _jet_case(model):
    nx, ny, nz = 64, 64, 512
    ins = inputs.jet(nx, ny, nz, 10.0, 1.0)          # lambda = 512/6 keeps the box periodic
    if model == "cg":
        rr, rb = inputs.two_fluid(ins, 1.0, 1.0, 0.01, 3)
        kw = dict(lattice=1, model=0, nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1.0, A=0.0675)  # sigma = 0.03
    else:
        rr, rb = inputs.two_fluid(ins, 1.0, 1.0, 0.01, 3)
        rr, rb = rr + 0.03, rb + 0.03
        kw = dict(lattice=1, model=2, nx=nx, ny=ny, nz=nz, G=0.9, rho0_psi=0.577)
    return C.Case("jet_" + model, kw, rr, rb)


@pytest.mark.parametrize("model", ["cg", "sc2c"])
def test_config3_jet_fp32_two_steps(orc, lbm, model):
    case = _jet_case(model)
    s = C.oracle_sim(orc, case)
    lat = C.gpu_lattice(lbm, case, lbm.FP32)
    lat.set_tiling(32, 8, 0)                          # the tuned launch shape of the cluster kernel
    s.step(2)
    lat.step(2)
    g, o = lat.pops().cpu().numpy(), s.pops()
    err = np.max(np.abs(g - o)) / np.max(np.abs(o))
    print(f"jet {model} 64x64x512 FP32, 2 steps: max |err| / max|f| {err:.2e}")
    assert err < 1e-6


@pytest.mark.parametrize("precision", [2, 3])
def test_config3_jet_16bit_against_fp32(lbm, precision):
    """Stated 16-bit accuracy (as in test_gpu_parity's F16_TOL) at full size, 50 steps."""
    case = _jet_case("cg")
    ref = C.gpu_lattice(lbm, case, lbm.FP32).step(50)
    lat = C.gpu_lattice(lbm, case, precision)
    t0, _ = lat.totals()
    lat.step(50)
    r32 = ref.moments(device=False)
    r16 = lat.moments(device=False)
    assert r16[4] == lbm.OK
    er = np.max(np.abs(r16[0] - r32[0])) / np.max(r32[0])
    dm = abs(r16[3]["mass_r"] - t0["mass_r"]) / t0["mass_r"]
    print(f"jet precision {precision}: rho err {er:.2e} of max, mass drift {dm:.2e}")
    tol = {2: (5e-4, 5e-5), 3: (5e-3, 1e-3)}[precision]
    assert er < tol[0] and dm < tol[1]


def _ligament_case(color_norm):
    nx, ny, nz = 96, 96, 768
    rr, rb = inputs.two_fluid(inputs.capsule(nx, ny, nz, 8.0, 640.0), 1.0, 1e-3, 0.01, 4)
    kw = dict(lattice=1, model=0, nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1e-3, tau_r=1.0, tau_b=0.51,
              A=0.0433, color_norm=color_norm)
    return C.Case("ligament", kw, rr, rb)


@pytest.mark.parametrize("color_norm", [0, 1])
def test_config4a_ligament_fp64_two_steps(orc, lbm, color_norm):
    """Ratio 1000 from a sharp interface is a violent start: within two steps the blue
    populations reach ~10^4 times the blue density (the oracle shows the same), so their
    sum cancels to 1e-3 and only FP64 storage and arithmetic keep it; the FP64 path is
    held to 1e-12 of the largest population on every population."""
    case = _ligament_case(color_norm)
    s = C.oracle_sim(orc, case)
    lat = C.gpu_lattice(lbm, case, lbm.FP64)
    s.step(2)
    lat.step(2)
    g, o = lat.pops().cpu().numpy(), s.pops()
    # a population's rounding is relative to the terms it is computed from; at this ratio
    # small populations are differences of terms up to the largest population (~25), so
    # the error is measured against that magnitude
    err = np.max(np.abs(g - o)) / np.max(np.abs(o))
    print(f"ligament 96x96x768 ratio 1000 color_norm {color_norm} FP64, 2 steps: max relative error {err:.2e}, "
          f"max|f| {np.max(np.abs(o)):.2e}")
    assert err < 1e-12


def test_config4b_emulsion_with_repulsion_fp32_two_steps(orc, lbm):
    n = 256
    ins, placed = inputs.emulsion(n, n, n, count=200, r_mean=10.0, r_spread=2.0, gap=3.0, seed=4)
    assert len(placed) == 200
    rr, rb = inputs.two_fluid(ins, 1.36, 1.36, 0.01, 5)
    kw = dict(lattice=1, model=0, nx=n, ny=n, nz=n, rho_r0=1.36, rho_b0=1.36, A=0.0518, rep_pi=0.012,
              rep_chi=2.0, grad_eps=1e-7)
    case = C.Case("emulsion", kw, rr, rb)
    s = C.oracle_sim(orc, case)
    lat = C.gpu_lattice(lbm, case, lbm.FP32)
    s.step(2)
    lat.step(2)
    rr_g, rb_g, u_g, tot, rc = lat.moments(device=False)
    orr, orb, ou, _ = s.moments()
    assert rc == lbm.OK
    scale = max(orr.max(), orb.max())
    er = np.max(np.abs(rr_g - orr) / np.maximum(np.abs(orr), 1e-3 * scale))
    eb = np.max(np.abs(rb_g - orb) / np.maximum(np.abs(orb), 1e-3 * scale))
    q_u = np.quantile(np.abs(u_g - ou).max(0), 0.99) / np.max(np.abs(ou))
    print(f"emulsion 256^3 with F_rep, FP32 2 steps: rho err {er:.2e}/{eb:.2e}, u 99% quantile {q_u:.2e} of max|u|")
    assert er < 1e-5 and eb < 1e-5 and q_u < 3e-5
