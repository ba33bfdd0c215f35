"""Ligament contraction (Sec. 3.3, Table contrParams): a capsule of radius R0 and length L
contracts under surface tension; its endpoint travels at u = sqrt(sigma / (rho_R R0)),
i.e. with slope -1 in x/R0 against t/t_cap, t_cap = sqrt(rho_R R0^3 / sigma), once the
start-up phase is over.  The paper's finding that the standard CG (without the enhanced
equilibrium terms) contracts markedly slower, and the enhanced one at the predicted
rate when the ambient fluid is nearly inviscid (tau_B = 0.55), is checked on the GPU path
(FP32) in the paper's 128 x 64 x 64 box (here with the ligament along z)."""
import math

import numpy as np
import pytest

from paper_2110_05197_gb300 import inputs
from tests import cases as C
from tests import observables as obs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():  # collected on CPU hosts only to be deselected
    pytest.skip("needs a CUDA device", allow_module_level=True)

# Table contrParams: set: (R0, L, sigma, rho_R, rho_B, tau_R, tau_B)
SETS = {1: (12.0, 112.0, 0.05, 2.0, 0.1, 1.0, 0.55),
        2: (10.0, 100.0, 0.0778, 1.99, 0.165, 1.0, 1.0),
        4: (10.0, 100.0, 0.0778, 1.99, 0.165, 1.0, 0.55)}


def _omega_interface(tau_r, tau_b):
    # Eqs. interpVisc, effRelax at rho^N = 0 (rho_R = rho_B there)
    nu_r, nu_b = (tau_r - 0.5) / 3, (tau_b - 0.5) / 3
    nu = 1.0 / (0.5 / nu_r + 0.5 / nu_b)
    return 1.0 / (3 * nu + 0.5)


def contraction_slope(lbm, set_id, enhanced, t_end=3.5, fit=(2.0, 3.5), every=10):
    R0, L, sigma, rho_r, rho_b, tau_r, tau_b = SETS[set_id]
    nx, ny, nz = 64, 64, 128
    A = 9.0 / 4.0 * sigma * _omega_interface(tau_r, tau_b)   # Eq. sigmaA
    rr, rb = inputs.two_fluid(inputs.capsule(nx, ny, nz, R0, L), rho_r, rho_b)
    kw = dict(lattice=1, model=0, nx=nx, ny=ny, nz=nz, rho_r0=rho_r, rho_b0=rho_b, tau_r=tau_r, tau_b=tau_b,
              A=A, enhanced_eq=int(enhanced))
    lat = C.gpu_lattice(lbm, C.Case("ligament", kw, rr, rb), lbm.FP32)
    t_cap = math.sqrt(rho_r * R0 ** 3 / sigma)
    ts, xs = [], []
    for s in range(0, int(t_end * t_cap) + every, every):
        if s:
            lat.step(every)
        m = lat.moments(device=False)
        assert m[4] == lbm.OK
        ts.append(s / t_cap)
        xs.append(obs.endpoint_along_z(m[0], m[1], (nz, ny, nx)) / R0)
    ts, xs = np.array(ts), np.array(xs)
    sel = (ts >= fit[0]) & (ts <= fit[1])
    slope = np.polyfit(ts[sel], xs[sel], 1)[0]
    print(f"set {set_id} enhanced={int(enhanced)}: x_end/R0 from {xs[0]:.3f} to {xs[-1]:.3f}, "
          f"slope over t/t_cap in {fit}: {slope:.3f} (analytical -1)")
    return slope


# The fit window: the endpoint first bulges and accelerates (start-up, up to t ~ 1.75 t_cap)
# and slows down as the drop rounds off (from t ~ 4 t_cap in set 1); in between its speed is
# constant.  Measured slopes (FP32): set 1 enhanced -0.94, standard -0.71; set 4 -0.90;
# set 2 -0.79.


def test_enhanced_equilibrium_matches_the_analytical_rate(lbm):
    s1 = contraction_slope(lbm, 1, True)
    s4 = contraction_slope(lbm, 4, True)
    assert abs(s1 + 1) < 0.12 and abs(s4 + 1) < 0.12


def test_standard_cg_contracts_slower(lbm):
    enh = contraction_slope(lbm, 1, True)
    std = contraction_slope(lbm, 1, False)
    assert std > enh + 0.15          # markedly slower (less negative slope)


def test_viscous_ambient_contracts_slower(lbm):
    # set 2 (tau_B = 1) against set 4 (tau_B = 0.55), otherwise equal
    assert contraction_slope(lbm, 2, True) > contraction_slope(lbm, 4, True) + 0.05
