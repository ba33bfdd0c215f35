"""The paper's benchmark observables per storage precision against the FP64 oracle: the
Laplace pressure jump of the static droplet (Sec. 3.1), the oscillation frequency of a
deformed droplet (Sec. 3.2) and the satellite-droplet mass of a broken jet (Sec. 3.4).
Each test runs the oracle once and the GPU path in FP64, FP32, FP16 and BF16 storage on
the same seeded input, prints the relative error of the observable and holds it to the
bound stated in ERR_BOUND (about three times the measured error).

Workloads: the D2Q9 128^2 droplet of radius 20 for its full 2000 steps; a 48^3 D3Q19
ellipsoid (semi-axes 13.2/11.4/11.4, ratio 10, tau 0.6) over 2400 steps, radius along x
every 20 steps; a 32x32x128 jet (radius 5, two wavelengths of 64, amplitude 1.5, tau 0.6,
sigma 0.03) broken after 1200 steps into two drops and two satellites.  The oscillation and
jet boxes are smaller than the paper-scale ones so that the oracle finishes in a minute."""
import numpy as np
import pytest

from paper_2110_05197_gb300 import inputs
from tests import cases as C
from tests import observables as obs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():  # collected on CPU hosts only to be deselected
    pytest.skip("needs a CUDA device", allow_module_level=True)

PRECISIONS = {0: "FP64", 1: "FP32", 2: "FP16", 3: "BF16"}
# stated relative error of each observable against the FP64 oracle, per storage precision
ERR_BOUND = {
    "laplace": {0: 1e-9, 1: 1e-5, 2: 1e-2, 3: 6e-2},
    "frequency": {0: 1e-9, 1: 2e-5, 2: 5e-3, 3: 1.5e-1},
    "satellite": {0: 1e-9, 1: 5e-6, 2: 2e-3, 3: 2e-3},
}


def _report(name, ref, vals):
    for prec, v in vals.items():
        err = abs(v - ref) / abs(ref)
        print(f"{name} {PRECISIONS[prec]}: {v:.6e} vs oracle {ref:.6e}, relative error {err:.2e}")
    for prec, v in vals.items():
        assert abs(v - ref) / abs(ref) < ERR_BOUND[name][prec], (name, PRECISIONS[prec])


def test_laplace_pressure_jump(orc, lbm):
    n = 128
    rr, rb = inputs.two_fluid(inputs.sphere(n, n, 1, 20.0), 1.0, 1.0, 0.0, 1)
    case = C.Case("laplace", dict(lattice=0, model=0, nx=n, ny=n, nz=1, rho_r0=1.0, rho_b0=1.0, A=1e-2), rr, rb)
    cs2 = 3 * (1 - 0.2) / 5          # D2Q9, alpha_R = alpha_B = 0.2 at ratio 1
    # Eqs. rhoin / rhoout pick the level eps = 1 - 0.1^n per field, and the largest n a
    # field reaches depends on its precision (the minority colour's floor), which would
    # change the averaging region; every field is measured at n = 3 (|rho^N| >= 0.999,
    # the bulk well away from the interface), and the per-field rule is printed beside it
    eps = 1 - 1e-3
    s = C.oracle_sim(orc, case).step(2000)
    o = s.moments()
    ref = obs.pressure_jump(o[0], o[1], cs2, cs2, eps)
    print(f"oracle: Delta P {ref:.6e} at eps = 0.999, {obs.pressure_jump(o[0], o[1], cs2, cs2):.6e} "
          f"at its own level 1 - {1 - obs.eps_level(obs.colour(o[0], o[1])):.0e}")
    vals = {}
    for prec in PRECISIONS:
        lat = C.gpu_lattice(lbm, case, prec).step(2000)
        m = lat.moments(device=False)
        assert m[4] == lbm.OK
        vals[prec] = obs.pressure_jump(m[0], m[1], cs2, cs2, eps)
        print(f"{PRECISIONS[prec]}: Delta P at its own level 1 - {1 - obs.eps_level(obs.colour(m[0], m[1])):.0e}: "
              f"{obs.pressure_jump(m[0], m[1], cs2, cs2):.6e}")
    _report("laplace", ref, vals)


def _osc_case():
    n = 48
    ins = inputs.ellipsoid(n, n, n, (13.2, 11.4, 11.4))
    rr, rb = inputs.two_fluid(ins, 1.0, 0.1, 0.0, 2)
    kw = dict(lattice=1, model=0, nx=n, ny=n, nz=n, rho_r0=1.0, rho_b0=0.1, tau_r=0.6, tau_b=0.6, A=0.03)
    return C.Case("oscillation", kw, rr, rb)


def _radius_history(sim_step, moments, shape, samples, every=20):
    out = []
    for _ in range(samples):
        sim_step(every)
        rr, rb = moments()
        out.append(obs.radius_along_x(rr, rb, shape))
    return np.array(out)


def test_oscillation_frequency(orc, lbm):
    case = _osc_case()
    n = case.kw["nx"]
    shape = (n, n, n)
    samples = 120
    s = C.oracle_sim(orc, case)
    skip = 10   # the first 200 steps: the sharp interface relaxing to its profile
    r_ref = _radius_history(s.step, lambda: s.moments()[:2], shape, samples)
    ref = obs.oscillation_frequency(r_ref[skip:], 20)
    vals = {}
    for prec in PRECISIONS:
        lat = C.gpu_lattice(lbm, case, prec)

        def mom():
            m = lat.moments(device=False)
            assert m[4] == lbm.OK
            return m[0], m[1]
        r = _radius_history(lat.step, mom, shape, samples)
        vals[prec] = obs.oscillation_frequency(r[skip:], 20)
        print(f"{PRECISIONS[prec]}: max |R - R_oracle| over the run {np.max(np.abs(r - r_ref)):.2e}")
    _report("frequency", ref, vals)


def _jet_case():
    nx, ny, nz = 32, 32, 128
    ins = inputs.jet(nx, ny, nz, 5.0, 1.5, 64.0)
    rr, rb = inputs.two_fluid(ins, 1.0, 1.0, 0.0, 3)
    kw = dict(lattice=1, model=0, nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1.0, tau_r=0.6, tau_b=0.6,
              A=2.25 * 0.03 / 0.6)   # sigma = (4/9) A / omega_eff = 0.03
    return C.Case("jet", kw, rr, rb)


def test_satellite_droplet_mass(orc, lbm):
    case = _jet_case()
    shape = (case.kw["nz"], case.kw["ny"], case.kw["nx"])
    s = C.oracle_sim(orc, case).step(1200)
    o = s.moments()
    ms = obs.droplet_masses(o[0], o[1], shape)
    assert len(ms) == 4, ms                      # two drops, two satellites
    ref = sum(ms[2:])
    vals = {}
    for prec in PRECISIONS:
        lat = C.gpu_lattice(lbm, case, prec).step(1200)
        m = lat.moments(device=False)
        assert m[4] == lbm.OK
        mg = obs.droplet_masses(m[0], m[1], shape)
        assert len(mg) == 4, (PRECISIONS[prec], mg)
        vals[prec] = sum(mg[2:])
    _report("satellite", ref, vals)
