"""The oracle against the independent NumPy transcription (tests/bruteforce.py) on tiny
lattices: 8 x 8 D2Q9 and 4 x 4 x 4 D3Q19, initial populations and 10 steps, every model
and flag combination (enhanced equilibrium on/off, colour normalisation, repulsion force
in both psi_rep forms, walls, body force, SC multiphase and two-component).

The two sum in different orders, so they agree to rounding: |bf - oracle| <= 1e-13 of the
largest population after 10 steps.  A plausible mistake in either (a dropped term, a
wrong sign, a transposed index, a wrong constant) shows up at 1e-4 or more."""
import numpy as np
import pytest

from paper_2110_05197_gb300 import inputs
from tests import bruteforce as bf

TOL = 1e-13


def _fields(d3, seed, ratio=1.0, walls=False):
    shape = (4, 4, 4) if d3 else (1, 8, 8)
    nz, ny, nx = shape
    n = nx * ny * nz
    a = inputs.uniform_pm1(seed, n, 0)
    b = inputs.uniform_pm1(seed, n, 1)
    rr = 0.55 + 0.4 * a                # both colours present everywhere, random interfaces
    rb = (0.55 - 0.4 * a) / ratio * (1 + 0.05 * b)
    solid = None
    if walls:
        solid = inputs.channel_walls(nx, ny, nz)
        rr = np.where(solid, 0.0, rr)
        rb = np.where(solid, 0.0, rb)
    u = 0.01 * np.stack([inputs.uniform_pm1(seed, n, 2), inputs.uniform_pm1(seed, n, 3),
                         inputs.uniform_pm1(seed, n, 4) if d3 else np.zeros(n)])
    if walls:
        u = np.where(solid[None, :], 0.0, u)
    return shape, rr, rb, u, solid


CG_CASES = {
    "plain": dict(A=1e-2),
    "standard_eq": dict(A=1e-2, enhanced=False),
    "ratio_norm": dict(A=5e-3, ratio=10.0, color_norm=True, tau_b=0.7),
    "visc_ratio": dict(A=5e-3, tau_r=1.3, tau_b=0.6, beta=0.5),
    "body": dict(A=1e-2, body=(1e-4, -2e-4, 5e-5)),
    "walls": dict(A=4e-3, walls=True, body=(1e-5, 0.0, 2e-6)),
    "rep": dict(A=5e-3, rep_pi=0.02, rep_chi=2.0, grad_eps=1e-9),
    "rep_printed": dict(A=5e-3, rep_pi=0.003, rep_chi=1.5, rep_printed=True, grad_eps=1e-9),
    "rep_walls": dict(A=5e-3, rep_pi=0.01, rep_chi=2.0, grad_eps=1e-9, walls=True),
}


def _oracle_kw(p: bf.Params, d3):
    nz, ny, nx = p.shape
    model = {"cg": 0, "sc_mp": 1, "sc_2c": 2}[p.model]
    return dict(lattice=1 if d3 else 0, model=model, nx=nx, ny=ny, nz=nz, rho_r0=p.rho_r0, rho_b0=p.rho_b0,
                alpha_b=p.alpha_b, tau_r=p.tau_r, tau_b=p.tau_b, A=p.A, beta=p.beta,
                enhanced_eq=int(p.enhanced), color_norm=int(p.color_norm), rep_pi=p.rep_pi, rep_chi=p.rep_chi,
                rep_psi_kind=int(p.rep_printed), grad_eps=p.grad_eps, G=p.G, rho0_psi=p.rho0,
                body_force=p.body)


def _compare(orc, p, d3, rr, rb, u, solid, steps=10):
    o = orc.OracleSim(orc.Params(**_oracle_kw(p, d3)))
    o.init(rr, rb, u, solid)
    b = bf.BruteForce(p).init(rr, rb, u)
    scale = np.max(np.abs(o.pops()))
    d0 = np.max(np.abs(o.pops() - b.pops())) / scale
    o.step(steps)
    b.step(steps)
    po, pb = o.pops(), b.pops()
    assert np.all(np.isfinite(po))
    d = np.max(np.abs(po - pb)) / np.max(np.abs(po))
    return d0, d


@pytest.mark.parametrize("d3", [False, True], ids=["d2q9_8x8", "d3q19_4x4x4"])
@pytest.mark.parametrize("name", list(CG_CASES))
def test_cg_matches_bruteforce(orc, d3, name):
    kw = dict(CG_CASES[name])
    ratio = kw.pop("ratio", 1.0)
    walls = kw.pop("walls", False)
    shape, rr, rb, u, solid = _fields(d3, seed=11 + len(name), ratio=ratio, walls=walls)
    p = bf.Params(d3=d3, model="cg", shape=shape, rho_b0=1.0 / ratio, solid=solid, **kw)
    if p.rep_pi:
        # the repulsion force is active on these random interfaces (not a trivial zero)
        b = bf.BruteForce(p).init(rr, rb, u)
        with np.errstate(divide="ignore", invalid="ignore"):
            rhoN = b.colour(b.f[0].sum(axis=0), b.f[1].sum(axis=0))
            assert np.abs(b.rep_force(rhoN, b.grad(rhoN))).max() > 1e-2 * p.rep_pi
    d0, d = _compare(orc, p, d3, rr, rb, u, solid)
    print(f"CG {name} d3={d3}: init {d0:.1e}, 10 steps {d:.1e}")
    assert d0 <= TOL and d <= TOL


SC_CASES = {
    "mp": dict(model="sc_mp", G=-5.0, rho0=1.0),
    "mp_body_walls": dict(model="sc_mp", G=-4.5, rho0=1.0, tau_r=0.8, body=(2e-5, 0.0, 1e-5), walls=True),
    "2c": dict(model="sc_2c", G=0.9, rho0=0.577, tau_b=0.8),
    "2c_body_walls": dict(model="sc_2c", G=0.9, rho0=0.577, tau_r=0.9, body=(1e-5, 2e-5, 0.0), walls=True),
}


@pytest.mark.parametrize("d3", [False, True], ids=["d2q9_8x8", "d3q19_4x4x4"])
@pytest.mark.parametrize("name", list(SC_CASES))
def test_sc_matches_bruteforce(orc, d3, name):
    kw = dict(SC_CASES[name])
    walls = kw.pop("walls", False)
    shape, rr, rb, u, solid = _fields(d3, seed=23 + len(name), walls=walls)
    if kw["model"] == "sc_mp":
        rr = np.where(rr > 0, 1.0 + 0.8 * (rr - 0.55) / 0.4, 0.0)  # liquid/gas mix around 1
        rb = None
    p = bf.Params(d3=d3, shape=shape, solid=solid, **kw)
    d0, d = _compare(orc, p, d3, rr, rb, u, solid)
    print(f"SC {name} d3={d3}: init {d0:.1e}, 10 steps {d:.1e}")
    assert d0 <= TOL and d <= TOL


def test_bruteforce_detects_a_planted_mistake(orc):
    """The comparison is sensitive: a transcription with the perturbation's B_i sign
    flipped is far outside the tolerance."""
    d3 = True
    shape, rr, rb, u, solid = _fields(d3, seed=5)
    p = bf.Params(d3=d3, model="cg", shape=shape, A=1e-2)
    good = bf.BruteForce(p).init(rr, rb, u)
    bad = bf.BruteForce(p).init(rr, rb, u)
    bad.L.B = -bad.L.B
    good.step(3)
    bad.step(3)
    o = orc.OracleSim(orc.Params(**_oracle_kw(p, d3)))
    o.init(rr, rb, u)
    o.step(3)
    po = o.pops()
    scale = np.max(np.abs(po))
    assert np.max(np.abs(po - good.pops())) / scale <= TOL
    assert np.max(np.abs(po - bad.pops())) / scale > 1e-6
