"""Pins of the oracle's per-node building blocks against facts the paper and the
mathematics fix: lattice isotropy, the moment identities of the constant tables, and the
moments of the equilibrium, Guo source, perturbation and recolouring operators.

Each check is a consequence of the definitions, not a re-typing of them: a dropped term,
a wrong sign or a transposed operand in the oracle changes a moment and fails here.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

LATTICES = [0, 1]  # D2Q9, D3Q19


def _frac(x):
    f = Fraction(x).limit_denominator(20000)
    assert abs(float(f) - x) < 1e-15
    return f


def _exact(c, v):
    return [_frac(x) for x in v]


@pytest.mark.parametrize("lat", LATTICES)
def test_velocity_set_and_weights(orc, lat):
    """Eq. speeds / weights: one rest vector, axis then diagonal group, opposites adjacent;
    sum w = 1, sum w c c = I/3, sum w c^4 = (1/9)(dd+dd+dd)."""
    c, w, *_ = orc.lattice_tables(lat)
    Q = 19 if lat == 1 else 9
    d = 3 if lat == 1 else 2
    assert c.shape == (Q, 3)
    assert (c[0] == 0).all()
    for i in range(1, Q, 2):
        assert (c[i] == -c[i + 1]).all()
    norms = (c * c).sum(1)
    assert sorted(set(norms[1:1 + 2 * d])) == [1] and set(norms[1 + 2 * d:]) == {2}
    assert len({tuple(v) for v in c}) == Q
    W = _exact(c, w)
    assert sum(W) == 1
    for a, b in itertools.product(range(d), repeat=2):
        assert sum(W[i] * int(c[i, a] * c[i, b]) for i in range(Q)) == (Fraction(1, 3) if a == b else 0)
    for a, b, g, h in itertools.product(range(d), repeat=4):
        lhs = sum(W[i] * int(c[i, a] * c[i, b] * c[i, g] * c[i, h]) for i in range(Q))
        rhs = Fraction(1, 9) * ((a == b) * (g == h) + (a == g) * (b == h) + (a == h) * (b == g))
        assert lhs == rhs
    # odd moments vanish
    for a in range(d):
        assert sum(W[i] * int(c[i, a]) for i in range(Q)) == 0


def _golden_constants():
    """tests/golden/d3q19_printed_constants.txt: the D3Q19 w, B, psi, xi values printed in
    Sec. 2.2 (Eqs. weights, perturbationOp, equiliCG)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "d3q19_printed_constants.txt")
    want = {}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        name, grp, val = line.split()
        want.setdefault(name, {})[int(grp)] = Fraction(val)
    return want


def test_d3q19_printed_values(orc):
    """The oracle's D3Q19 tables equal the values printed with Eqs. weights,
    perturbationOp and equiliCG (golden fixture)."""
    c, w, B, psi, xi = orc.lattice_tables(1)
    grp = [0] + [1] * 6 + [2] * 12
    want = _golden_constants()
    assert set(want) == {"w", "B", "psi", "xi"}
    for name, arr in (("w", w), ("B", B), ("psi", psi), ("xi", xi)):
        for i in range(19):
            assert _frac(arr[i]) == want[name][grp[i]], (name, i)


@pytest.mark.parametrize("lat", LATTICES)
def test_perturbation_table_moments(orc, lat):
    """sum_i B_i = 1/3 = sum_i w_i (c_i.n)^2 for unit n, and sum_i B_i c c = I/3, so the
    perturbation bracket carries no mass and has the stress (2/9)(nn - I)."""
    c, w, B, *_ = orc.lattice_tables(lat)
    Q, d = len(w), (3 if lat == 1 else 2)
    Bx = _exact(c, B)
    assert sum(Bx) == Fraction(1, 3)
    for a, b in itertools.product(range(d), repeat=2):
        assert sum(Bx[i] * int(c[i, a] * c[i, b]) for i in range(Q)) == (Fraction(1, 3) if a == b else 0)


@pytest.mark.parametrize("lat", LATTICES)
def test_enhanced_table_moments(orc, lat):
    """psi_i, xi_i: sum psi + 2 sum xi c_x^2 = 0 (no mass), sum psi c c = 0, and
    sum xi c^4 = (1/2)(dd+dd+dd) -- the conditions behind the second moment of Eq. equiliCG."""
    c, w, B, psi, xi = orc.lattice_tables(lat)
    Q, d = len(w), (3 if lat == 1 else 2)
    P, X = _exact(c, psi), _exact(c, xi)
    assert sum(P) == -3
    assert sum(X[i] * int(c[i, 0] ** 2) for i in range(Q)) == Fraction(3, 2)
    for a, b in itertools.product(range(d), repeat=2):
        assert sum(P[i] * int(c[i, a] * c[i, b]) for i in range(Q)) == 0
    for a, b, g, h in itertools.product(range(d), repeat=4):
        lhs = sum(X[i] * int(c[i, a] * c[i, b] * c[i, g] * c[i, h]) for i in range(Q))
        rhs = Fraction(1, 2) * ((a == b) * (g == h) + (a == g) * (b == h) + (a == h) * (b == g))
        assert lhs == rhs


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("alpha", [0.2, 0.55, 0.92, 0.9992])
def test_phi_moments(orc, lat, alpha):
    """Eq. phi: sum phi = 1, sum phi c c = c_s^2 I with c_s^2 = (1-alpha)/2 (Eq. CGpressure,
    D3Q19) or 3(1-alpha)/5 (D2Q9)."""
    c, w, *_ = orc.lattice_tables(lat)
    ph = orc.phi(lat, alpha)
    cs2 = (1 - alpha) / 2 if lat == 1 else 3 * (1 - alpha) / 5
    assert abs(ph.sum() - 1) < 1e-15
    M2 = np.einsum("i,ia,ib->ab", ph, c, c)
    d = 3 if lat == 1 else 2
    assert np.allclose(M2[:d, :d], cs2 * np.eye(d), atol=1e-15, rtol=0)


@pytest.mark.parametrize("lat", LATTICES)
def test_phi_reduces_to_weights(orc, lat):
    """alpha = 1/3 (D3Q19) or 4/9 (D2Q9) makes phi_i = w_i: the CG equilibrium becomes the
    standard one (Eq. equiliSC)."""
    c, w, *_ = orc.lattice_tables(lat)
    alpha = 1 / 3 if lat == 1 else 4 / 9
    assert np.allclose(orc.phi(lat, alpha), w, atol=1e-16, rtol=0)


def _rand_state(seed, d):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-0.05, 0.05, 3)
    g = rng.uniform(-0.2, 0.2, 3)
    if d == 2:
        u[2] = 0.0
        g[2] = 0.0
    return rng, u, g


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("enh", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_cg_equilibrium_moments(orc, lat, enh, seed):
    """Eq. equiliCG: sum f^eq = rho_k, sum f^eq c = rho_k u, and
    sum f^eq c c = p_k I + rho_k u u + nubar[(u.grad) I + u grad^T + grad u^T]
    (the enhanced part only when enabled)."""
    d = 3 if lat == 1 else 2
    c, *_ = orc.lattice_tables(lat)
    rng, u, g = _rand_state(seed, d)
    rho, alpha, nubar = rng.uniform(0.1, 3), rng.uniform(0.1, 0.95), rng.uniform(0.02, 0.5)
    feq = orc.cg_equilibrium(lat, rho, alpha, u, g, nubar, enh)
    cs2 = (1 - alpha) / 2 if lat == 1 else 3 * (1 - alpha) / 5
    assert abs(feq.sum() - rho) < 1e-14
    assert np.allclose(feq @ c, rho * u, atol=1e-15)
    M2 = np.einsum("i,ia,ib->ab", feq, c, c)
    want = cs2 * rho * np.eye(3) + rho * np.outer(u, u)
    if enh:
        want += nubar * (np.dot(u, g) * np.eye(3) + np.outer(u, g) + np.outer(g, u))
    assert np.allclose(M2[:d, :d], want[:d, :d], atol=1e-14, rtol=0)


@pytest.mark.parametrize("lat", LATTICES)
def test_sc_equilibrium_moments(orc, lat):
    """Eq. equiliSC: moments rho, rho u, rho/3 I + rho u u."""
    d = 3 if lat == 1 else 2
    c, *_ = orc.lattice_tables(lat)
    rng, u, _ = _rand_state(11, d)
    feq = orc.sc_equilibrium(lat, 1.7, u)
    assert abs(feq.sum() - 1.7) < 1e-14
    assert np.allclose(feq @ c, 1.7 * u, atol=1e-15)
    M2 = np.einsum("i,ia,ib->ab", feq, c, c)
    want = 1.7 / 3 * np.eye(3) + 1.7 * np.outer(u, u)
    assert np.allclose(M2[:d, :d], want[:d, :d], atol=1e-14)


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("omega", [0.6, 1.0, 1.7])
def test_guo_source_moments(orc, lat, omega):
    """Eq. source: sum S = 0, sum S c = (1 - omega/2) F, sum S c c = (1 - omega/2)(u F^T + F u^T)."""
    d = 3 if lat == 1 else 2
    c, *_ = orc.lattice_tables(lat)
    rng, u, F = _rand_state(5, d)
    S = orc.guo_source(lat, u, F, omega)
    k = 1 - omega / 2
    assert abs(S.sum()) < 1e-15
    assert np.allclose(S @ c, k * F, atol=1e-15)
    M2 = np.einsum("i,ia,ib->ab", S, c, c)
    want = k * (np.outer(u, F) + np.outer(F, u))
    assert np.allclose(M2[:d, :d], want[:d, :d], atol=1e-15)


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("seed", range(3))
def test_perturbation_moments(orc, lat, seed):
    """Eq. perturbationOp (reading A|grad rho^N|[..] on the total): no mass, no momentum,
    second moment (2/9) A |g| (n n^T - I); zero when |g| <= eps."""
    d = 3 if lat == 1 else 2
    c, *_ = orc.lattice_tables(lat)
    rng, _, g = _rand_state(seed + 20, d)
    A = 0.013
    dP = orc.perturbation(lat, g, A)
    gn = np.linalg.norm(g)
    n = g / gn
    assert abs(dP.sum()) < 1e-16
    assert np.allclose(dP @ c, 0, atol=1e-17)
    M2 = np.einsum("i,ia,ib->ab", dP, c, c)
    want = 2 / 9 * A * gn * (np.outer(n, n) - np.eye(3))
    assert np.allclose(M2[:d, :d], want[:d, :d], atol=1e-16)
    assert np.all(orc.perturbation(lat, g, A, eps=2 * gn) == 0)


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("seed", range(3))
def test_recolor_moments(orc, lat, seed):
    """Eqs. recoloringOpR/B with cosphi: f^R + f^B = f*, sum f^R = rho_R, and the colour
    flux sum (f^R - rho_R/rho f*) c = beta rho_R rho_B/rho^2 sum_k rho_k K_k n with
    K = 2 phi_axis + (2d-... ) phi_diag/sqrt2 from the direction sums."""
    d = 3 if lat == 1 else 2
    c, *_ = orc.lattice_tables(lat)
    rng, u, g = _rand_state(seed + 40, d)
    rr, rb = rng.uniform(0.05, 2), rng.uniform(0.05, 2)
    ar, ab = 0.7, 0.2
    nubar = 0.1
    fstar = (orc.cg_equilibrium(lat, rr, ar, u, g, nubar) + orc.cg_equilibrium(lat, rb, ab, u, g, nubar)
             + rng.uniform(-1e-3, 1e-3, len(c)) * 0)
    beta = 0.7
    fr, fb = orc.recolor(lat, fstar, rr, rb, ar, ab, g, beta)
    rho = rr + rb
    assert np.allclose(fr + fb, fstar, atol=1e-15)
    assert abs(fr.sum() - rr) < 1e-14 and abs(fb.sum() - rb) < 1e-14
    n = g / np.linalg.norm(g)
    ndiag = 8 if lat == 1 else 4

    def K(alpha):
        ph = orc.phi(lat, alpha)
        return 2 * ph[1] + ndiag * ph[-1] / np.sqrt(2)

    flux = (fr - rr / rho * fstar) @ c
    want = beta * rr * rb / rho ** 2 * (rr * K(ar) + rb * K(ab)) * n
    assert np.allclose(flux[:d], want[:d], atol=1e-15)
    # without a gradient the split is by density only
    fr0, _ = orc.recolor(lat, fstar, rr, rb, ar, ab, np.zeros(3), beta)
    assert np.allclose(fr0, rr / rho * fstar, atol=1e-16)
