"""Pins of the oracle's multicomponent Shan-Chen model with multirange potentials (Sec. 2.1,
Eqs. benziforces, doublebeltattractiveforce, doublebeltrepulsionforce, pweights,
doublebeltrepulsionforce2): the belt weights' isotropy, the reduction to the two-component
model, the independent NumPy transcription on a 6^3 lattice (distance-2 neighbours
distinct), and conservation on a periodic box."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2110_05197_gb300 import inputs
from tests import bruteforce as bf

# Table dropcolParams set 1 (SC): G^a = (-9, -8), G^r = (8.1, 7.1), G_AB = 0.405, rho_0 = 0.83
BENZI = dict(Ga=(-9.0, -8.0), Gr=(8.1, 7.1), G=0.405, rho0_psi=0.83)


def test_belt_vectors_and_weights(orc):
    c, p = orc.mr_vectors()
    assert len(c) == 93 and tuple(c[0]) == (0, 0, 0) and p[0] == 0.0
    r2 = (c ** 2).sum(1)
    assert [int((r2 == k).sum()) for k in (0, 1, 2, 3, 4, 5, 6, 8)] == [1, 6, 12, 8, 6, 24, 24, 12]
    assert len({tuple(v) for v in c}) == 93
    # the weights as exact fractions (Eq. pweights)
    P = {1: Fraction(4, 135), 2: Fraction(1, 63), 3: Fraction(2, 315), 4: Fraction(5, 1512),
         5: Fraction(1, 945), 6: Fraction(1, 1890), 8: Fraction(1, 15120)}
    for v, w in zip(c[1:], p[1:]):
        assert w == float(P[int((v ** 2).sum())])
    # second-order isotropy sum p c_a c_b = delta_ab / 3, fourth-order isotropy
    # sum p c_x^4 = 3 sum p c_x^2 c_y^2, vanishing odd moments -- exactly
    for a in range(3):
        for b in range(3):
            s = sum(P[int((v ** 2).sum())] * int(v[a]) * int(v[b]) for v in c[1:])
            assert s == (Fraction(1, 3) if a == b else 0)
        assert sum(P[int((v ** 2).sum())] * int(v[a]) for v in c[1:]) == 0
    s4 = sum(P[int((v ** 2).sum())] * int(v[0]) ** 4 for v in c[1:])
    s22 = sum(P[int((v ** 2).sum())] * int(v[0]) ** 2 * int(v[1]) ** 2 for v in c[1:])
    assert s4 == 3 * s22


def _fields(seed, n=6):
    N = n ** 3
    a = inputs.uniform_pm1(seed, N, 0)
    rr = 0.77 + 0.55 * a                     # both species everywhere, total ~1.36
    rb = (1.36 - rr) * (1 + 0.05 * inputs.uniform_pm1(seed, N, 1))
    u = 0.01 * np.stack([inputs.uniform_pm1(seed, N, k) for k in (2, 3, 4)])
    return rr, rb, u


def _oracle(orc, n=6, solid=None, **kw):
    p = orc.Params(lattice=1, model=orc.SC_MR, nx=n, ny=n, nz=n, **kw)
    return orc.OracleSim(p)


@pytest.mark.parametrize("case", ["benzi", "benzi_tau_body_walls"])
def test_multirange_matches_bruteforce(orc, case):
    n = 6
    rr, rb, u = _fields(31)
    kw = dict(BENZI)
    solid = None
    if case != "benzi":
        kw.update(tau_r=0.9, tau_b=0.7, body_force=(1e-5, -2e-5, 3e-6))
        solid = inputs.channel_walls(n, n, n)
        rr, rb = np.where(solid, 0.0, rr), np.where(solid, 0.0, rb)
        u = np.where(solid[None, :], 0.0, u)
    o = _oracle(orc, **kw)
    o.init(rr, rb, u, solid)
    b = bf.BruteForce(bf.Params(d3=True, model="sc_mr", shape=(n, n, n), Ga=kw["Ga"], Gr=kw["Gr"], G=kw["G"],
                                rho0=kw["rho0_psi"], tau_r=kw.get("tau_r", 1.0), tau_b=kw.get("tau_b", 1.0),
                                body=kw.get("body_force", (0.0, 0.0, 0.0)), solid=solid)).init(rr, rb, u)
    # the force is far from zero on these fields
    F = o.force()
    fluid = np.ones(n ** 3, bool) if solid is None else solid == 0
    assert np.abs(F[:, fluid]).max() > 1e-2
    o.step(10)
    b.step(10)
    po, pb = o.pops(), b.pops()
    d = np.max(np.abs(po - pb)) / np.max(np.abs(po))
    print(f"multirange {case}: oracle vs brute force after 10 steps {d:.1e}")
    assert np.all(np.isfinite(po)) and d <= 1e-13


def test_bruteforce_sees_a_flipped_repulsion(orc):
    rr, rb, u = _fields(32)
    o = _oracle(orc, **BENZI)
    o.init(rr, rb, u)
    o.step(3)
    good = bf.BruteForce(bf.Params(d3=True, model="sc_mr", shape=(6, 6, 6), Ga=BENZI["Ga"], Gr=BENZI["Gr"],
                                   G=BENZI["G"], rho0=BENZI["rho0_psi"])).init(rr, rb, u).step(3)
    bad = bf.BruteForce(bf.Params(d3=True, model="sc_mr", shape=(6, 6, 6), Ga=BENZI["Ga"],
                                  Gr=(-BENZI["Gr"][0], -BENZI["Gr"][1]), G=BENZI["G"],
                                  rho0=BENZI["rho0_psi"])).init(rr, rb, u).step(3)
    scale = np.max(np.abs(o.pops()))
    assert np.max(np.abs(o.pops() - good.pops())) / scale <= 1e-13
    assert np.max(np.abs(o.pops() - bad.pops())) / scale > 1e-6


def test_reduces_to_two_component_without_self_couplings(orc):
    n = 8
    rr, rb = inputs.two_fluid(inputs.sphere(n, n, n, 2.5), 1.0, 1.0, 0.01, 4)
    rr, rb = rr + 0.03, rb + 0.03
    kw = dict(lattice=1, nx=n, ny=n, nz=n, G=0.9, rho0_psi=0.577, tau_b=0.8)
    a = orc.OracleSim(orc.Params(model=orc.SC_2C, **kw))
    b = orc.OracleSim(orc.Params(model=orc.SC_MR, **kw))
    a.init(rr, rb)
    b.init(rr, rb)
    a.step(20)
    b.step(20)
    assert np.max(np.abs(a.pops() - b.pops())) <= 1e-14 * np.max(np.abs(a.pops()))


def test_printed_cross_coupling_does_not_demix(orc):
    """With this model's lattice weights (sum w c c = I/3) the printed G_AB = 0.405 and
    rho_0 = 0.83 give G_AB rho / rho_0^2 = 0.8 < 2, below the demixing threshold of the cross
    force, and the self-couplings' net -0.9 is far below a multiphase SC's critical value:
    an A-rich slab dissolves (the reading behind the factor 3 on G_AB in the GPU cases)."""
    n = 16
    x = inputs.grid(n, 4, 4)[0]
    slab = (x >= 4) & (x < 12)
    rr = np.where(slab, 1.18, 0.18)
    rb = np.where(slab, 0.18, 1.18)
    o = orc.OracleSim(orc.Params(lattice=1, model=orc.SC_MR, nx=n, ny=4, nz=4, **BENZI))
    o.init(rr, rb)
    o.step(1000)
    r = o.moments()[0]
    assert np.ptp(r) < 0.05
    o = orc.OracleSim(orc.Params(lattice=1, model=orc.SC_MR, nx=n, ny=4, nz=4, **dict(BENZI, G=3 * BENZI["G"])))
    o.init(rr, rb)
    o.step(1000)
    line = o.moments()[0].reshape(4, 4, n)[0, 0]
    assert line[7] > 1.3 and line[0] < 0.15   # demixed: A-rich centre, A-poor far side


def test_multirange_conserves_mass_and_momentum(orc):
    n = 12
    x = inputs.grid(n, n, n)[0]
    slab = (x >= 3) & (x < 9)
    rr = np.where(slab, 1.18, 0.18) * (1 + 0.01 * inputs.uniform_pm1(6, n ** 3, 0))
    rb = np.where(slab, 0.18, 1.18) * (1 + 0.01 * inputs.uniform_pm1(6, n ** 3, 1))
    o = _oracle(orc, n=n, **dict(BENZI, G=3 * BENZI["G"]))
    o.init(rr, rb)
    t0 = o.totals()
    o.step(50)
    t1 = o.totals()
    for m in ("mass_r", "mass_b"):
        assert abs(t1[m] - t0[m]) <= 1e-12 * t0[m]
    for m in ("mom_x", "mom_y", "mom_z"):
        assert abs(t1[m] - t0[m]) <= 1e-12 * t0["mass_r"]
    # the slabs stay separated: the majority species keeps its side
    r, b, _, _ = o.moments()
    assert r[slab].mean() > 1.0 and b[~slab].mean() > 1.0
