"""Pins of the full oracle step against physics the paper and textbook LBM fix:
conservation laws, reduction to plain BGK, the shear-wave decay rate, single- and
two-phase Poiseuille flow, Laplace's law (Eq. YoungLaplace, sigma from Eq. sigmaA), the SC
coexistence densities the paper prints (Sec. 3.2 / 3.3 tables) and the geometry of the CG
repulsion force (Eq. repForce).
"""
import numpy as np
import pytest

from paper_2110_05197_gb300 import inputs


def _sim(orc, **kw):
    return orc.OracleSim(orc.Params(**kw))


# ---------------------------------------------------------------- conservation

@pytest.mark.parametrize("ratio", [1.0, 10.0])
def test_cg_conserves_colour_mass_and_momentum(orc, ratio):
    """Per-colour mass (recolouring keeps rho_k per node) and total momentum (perturbation
    and recolouring carry none) are conserved to rounding on a periodic box."""
    n = 14
    rr, rb = inputs.two_fluid(inputs.ellipsoid(n, n, n, (5, 4, 4)), 1.0, 1.0 / ratio, 0.01, 3)
    s = _sim(orc, nx=n, ny=n, nz=n, rho_r0=1.0, rho_b0=1.0 / ratio, A=5e-3, tau_r=1.0, tau_b=0.7)
    s.init(rr, rb)
    t0 = s.totals()
    s.step(60)
    t1 = s.totals()
    assert abs(t1["mass_r"] - t0["mass_r"]) < 1e-12 * t0["mass_r"]
    assert abs(t1["mass_b"] - t0["mass_b"]) < 1e-12 * t0["mass_b"]
    for k in ("mom_x", "mom_y", "mom_z"):
        assert abs(t1[k]) < 1e-12
    assert t1["max_u"] > 1e-5  # the droplet does move


def test_sc_multiphase_conserves_mass_and_momentum(orc):
    """SC pair force sum_x psi(x) sum_i w_i psi(x+c_i) c_i is antisymmetric: zero total."""
    n = 12
    rr, _ = inputs.two_fluid(inputs.sphere(n, n, n, 4), 2.0, 0.0, 0.0)
    rr = np.where(rr > 0, 2.0, 0.15) * (1 + 0.01 * inputs.uniform_pm1(9, n ** 3))
    s = _sim(orc, model=orc.SC_MP, nx=n, ny=n, nz=n, G=-5.0, rho0_psi=1.0)
    s.init(rr)
    t0 = s.totals()
    s.step(60)
    t1 = s.totals()
    assert abs(t1["mass_r"] - t0["mass_r"]) < 1e-12 * t0["mass_r"]
    for k in ("mom_x", "mom_y", "mom_z"):
        assert abs(t1[k]) < 1e-12
    assert t1["max_u"] > 1e-4


def test_sc_two_component_conserves(orc):
    n = 12
    rr, rb = inputs.two_fluid(inputs.sphere(n, n, n, 4), 1.0, 1.0, 0.01, 4)
    s = _sim(orc, model=orc.SC_2C, nx=n, ny=n, nz=n, G=0.9, rho0_psi=0.577, tau_r=1.0, tau_b=1.0)
    s.init(rr + 0.02, rb + 0.02)
    t0 = s.totals()
    s.step(60)
    t1 = s.totals()
    assert abs(t1["mass_r"] - t0["mass_r"]) < 1e-12 * t0["mass_r"]
    assert abs(t1["mass_b"] - t0["mass_b"]) < 1e-12 * t0["mass_b"]
    for k in ("mom_x", "mom_y", "mom_z"):
        assert abs(t1[k]) < 1e-12


# ---------------------------------------------------------------- textbook BGK

def _textbook_bgk(c, w, rho, u, tau, steps, shape):
    """Plain single-population BGK with pull streaming on a periodic box (a textbook
    routine, independent of the oracle): f^eq = rho w (1 + 3cu + 4.5(cu)^2 - 1.5u^2)."""
    nz, ny, nx = shape
    Q = len(w)

    def feq(rho, u):
        cu = np.einsum("ia,a...->i...", c.astype(float), u)
        uu = (u * u).sum(0)
        return rho[None] * w[:, None, None, None] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * uu[None])

    f = feq(rho, u)
    for _ in range(steps):
        rho = f.sum(0)
        u = np.einsum("ia,i...->a...", c.astype(float), f) / rho
        f = f - (f - feq(rho, u)) / tau
        f = np.stack([np.roll(f[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2)) for i in range(Q)])
    return f


@pytest.mark.parametrize("lat", [0, 1])
def test_cg_reduces_to_bgk(orc, lat):
    """CG with A = 0, beta = 0, equal alpha = 1/3 (4/9 in 2D) and the standard equilibrium:
    the total population evolves exactly as plain BGK with rho = rho_R + rho_B."""
    shape = (4, 5, 6) if lat == 1 else (1, 7, 8)
    nz, ny, nx = shape
    N = nx * ny * nz
    alpha = 1 / 3 if lat == 1 else 4 / 9
    rng = np.random.default_rng(1)
    rr = 1 + 0.05 * rng.standard_normal(N)
    rb = 0.5 + 0.05 * rng.standard_normal(N)
    u = 0.02 * rng.standard_normal((3, N))
    if lat == 0:
        u[2] = 0
    s = _sim(orc, lattice=lat, nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1.0, alpha_b=alpha, A=0.0,
             beta=0.0, enhanced_eq=0, tau_r=0.8, tau_b=0.8)
    s.init(rr, rb, u)
    s.step(15)
    tot = s.pops().sum(0)
    c, w, *_ = orc.lattice_tables(lat)
    ref = _textbook_bgk(c, w, (rr + rb).reshape(shape), u.reshape(3, *shape), 0.8, 15, shape)
    assert np.max(np.abs(tot - ref.reshape(len(w), N))) < 1e-14


@pytest.mark.parametrize("lat", [0, 1])
def test_sc_without_coupling_is_bgk(orc, lat):
    shape = (4, 5, 6) if lat == 1 else (1, 7, 8)
    nz, ny, nx = shape
    N = nx * ny * nz
    rng = np.random.default_rng(2)
    rho = 1 + 0.05 * rng.standard_normal(N)
    u = 0.02 * rng.standard_normal((3, N))
    if lat == 0:
        u[2] = 0
    s = _sim(orc, lattice=lat, model=orc.SC_MP, nx=nx, ny=ny, nz=nz, G=0.0, tau_r=0.7)
    s.init(rho, None, u)
    s.step(15)
    c, w, *_ = orc.lattice_tables(lat)
    ref = _textbook_bgk(c, w, rho.reshape(shape), u.reshape(3, *shape), 0.7, 15, shape)
    assert np.max(np.abs(s.pops()[0] - ref.reshape(len(w), N))) < 1e-14


# ---------------------------------------------------------------- analytic flows

@pytest.mark.parametrize("tau", [0.8, 1.2])
def test_shear_wave_decay(orc, tau):
    """u_x = U sin(k y) decays as exp(-nu k^2 t), nu = (tau - 1/2)/3 (single colour, CG
    with the enhanced equilibrium)."""
    ny, steps = 32, 300
    u = inputs.shear_wave_velocity(1, ny, 1, 1e-4)
    s = _sim(orc, nx=1, ny=ny, nz=1, rho_r0=1.0, rho_b0=1.0, A=1e-2, tau_r=tau, tau_b=tau)
    s.init(np.ones(ny), np.zeros(ny), u)
    s.step(steps)
    _, _, uu, _ = s.moments()
    y = np.arange(ny)
    amp = 2 * np.mean(uu[0] * np.sin(2 * np.pi * y / ny))
    nu = (tau - 0.5) / 3
    k = 2 * np.pi / ny
    assert abs(amp / 1e-4 - np.exp(-nu * k * k * steps)) < 2e-3


def _poiseuille(orc, tau, ny=18, steps=8000, F=1e-6):
    solid = inputs.channel_walls(1, ny, 1)
    s = _sim(orc, nx=1, ny=ny, nz=1, rho_r0=1.0, rho_b0=1.0, tau_r=tau, tau_b=tau, A=0.0,
             body_force=(F, 0.0, 0.0))
    s.init(np.where(solid, 0.0, 1.0), np.zeros(ny), None, solid)
    s.step(steps)
    _, _, u, _ = s.moments()
    y = np.arange(ny, dtype=float)
    nu = (tau - 0.5) / 3
    exact = F / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    fl = solid == 0
    return np.linalg.norm(u[0][fl] - exact[fl]) / np.linalg.norm(exact[fl])


def test_poiseuille_magic_tau(orc):
    """Halfway bounce-back + Guo forcing + BGK reproduce the parabola exactly (to the
    convergence of the run) at (tau - 1/2)^2 = 3/16."""
    assert _poiseuille(orc, 0.5 + np.sqrt(3) / 4) < 1e-6


def test_poiseuille_tau_one(orc):
    assert _poiseuille(orc, 1.0) < 1e-2


def test_layered_two_phase_poiseuille(orc):
    """Red core |y - yc| < a between blue layers, equal densities, viscosity ratio 3:
    piecewise parabola u_B = F(h^2 - y^2)/(2 mu_B), u_R = F(a^2 - y^2)/(2 mu_R) + F(h^2 - a^2)/(2 mu_B)."""
    ny, F, a = 34, 1e-6, 8.0
    solid = inputs.channel_walls(1, ny, 1)
    y = np.arange(ny, dtype=float)
    yc = (ny - 1) / 2
    h = (ny - 2) / 2
    core = np.abs(y - yc) < a
    rr = np.where(core & (solid == 0), 1.0, 0.0)
    rb = np.where(~core & (solid == 0), 1.0, 0.0)
    tr, tb = 1.4, 0.8
    s = _sim(orc, nx=1, ny=ny, nz=1, rho_r0=1.0, rho_b0=1.0, tau_r=tr, tau_b=tb, A=1e-3,
             body_force=(F, 0.0, 0.0))
    s.init(rr, rb, None, solid)
    s.step(12000)
    _, _, u, t = s.moments()
    mr, mb = (tr - 0.5) / 3, (tb - 0.5) / 3
    yy = y - yc
    exact = np.where(np.abs(yy) < a, F * (a * a - yy ** 2) / (2 * mr) + F * (h * h - a * a) / (2 * mb),
                     F * (h * h - yy ** 2) / (2 * mb))
    fl = solid == 0
    err = np.linalg.norm(u[0][fl] - exact[fl]) / np.linalg.norm(exact[fl])
    assert err < 0.05
    assert abs(t[0] - rr.sum()) < 1e-10


# ---------------------------------------------------------------- Laplace (2D)

def _laplace_2d(orc, R, n=64, steps=1500, A=1e-2):
    rr, rb = inputs.two_fluid(inputs.sphere(n, n, 1, R), 1.0, 1.0)
    s = _sim(orc, lattice=0, nx=n, ny=n, nz=1, rho_r0=1.0, rho_b0=1.0, A=A, tau_r=1.0, tau_b=1.0)
    s.init(rr, rb)
    s.step(steps)
    r, b, u, t = s.moments()
    col = (r - b) / (r + b)
    # Eqs. rhoin / rhoout: eps = 1 - 0.1^n with the largest n <= 10 both sides still reach
    eps = None
    for k in range(10, 0, -1):
        e = 1 - 0.1 ** k
        if (col >= e).any() and (col <= -e).any():
            eps = e
            break
    rho_in = r[col >= eps].mean()
    rho_out = b[col <= -eps].mean()
    cs2 = 3 * (1 - 0.2) / 5
    dP = cs2 * (rho_in - rho_out)
    Reff = np.sqrt(((1 + col) / 2).sum() / np.pi)
    return dP * Reff, t


def test_laplace_2d(orc):
    """2D Young-Laplace over R = 10 ... 30: Delta P * R is the surface tension, constant
    across radii within 5%, and at R = 20 within 5% of sigma_th = (4/9) A / omega_eff =
    4.44e-3 (A = 1e-2, omega = 1; the paper's own error at R = 20 is a few per cent, Fig.
    vardens).  Larger drops relax over about R^2 / nu steps, so R = 20 and 30 run 8000 and
    9000 steps (96^2 box).  Measured errors: +2.8%, +0.4%, -0.4% at R = 10, 14, 18 and
    +0.9%, -0.3% at R = 20, 30."""
    sig_th = 4 / 9 * 1e-2
    vals = {}
    for R, n, steps in ((10, 64, 1500), (14, 64, 1500), (18, 64, 1500), (20, 96, 8000), (30, 96, 9000)):
        sig, t = _laplace_2d(orc, R, n=n, steps=steps)
        vals[R] = sig
        print("Laplace 2D R=%d (%d^2, %d steps) sigma_cal=%.5e, error %+.4f" % (R, n, steps, sig, sig / sig_th - 1))
        assert t[6] < 1e-3  # spurious currents stay small
    v = np.array(list(vals.values()))
    assert np.ptp(v) / v.mean() < 0.05
    assert abs(vals[20] - sig_th) / sig_th < 0.05


# ---------------------------------------------------------------- Shan-Chen coexistence

def _mechanical_stability(G):
    """Flat-interface coexistence of the SC equation of state p = rho/3 + (G/6) psi^2 with
    psi = 1 - exp(-rho): equal pressure and int_{rho_g}^{rho_l} (p_0 - p) psi'/psi^(1+eps) drho
    = 0, the mechanical-stability condition of the discrete pseudopotential pressure tensor
    (Shan, PRE 77 066702, 2008; Li, Luo & Li, PRE 86 016709, 2012), with eps = 0 for Guo's
    forcing scheme."""
    from scipy.integrate import quad
    from scipy.optimize import fsolve
    psi = lambda r: 1 - np.exp(-r)
    p = lambda r: r / 3 + G / 6 * psi(r) ** 2

    def eqs(v):
        g, l = v
        return [p(l) - p(g),
                quad(lambda r: (p(g) - p(r)) * np.exp(-r) / psi(r), g, l, limit=200)[0]]
    g, l = fsolve(eqs, [0.1, 2.0], xtol=1e-13)
    return l, g


@pytest.mark.parametrize("G", [-5.0, -5.4])
def test_sc_coexistence_mechanical_stability(orc, G):
    """A flat liquid/gas interface relaxes to the mechanical-stability coexistence densities
    of the SC equation of state (Eqs. interactionforceMP, pseudopotential with rho_0 = 1,
    Guo forcing).  At G = -5 this gives (1.888, 0.119); the paper's table prints (1.99,
    0.165), which no flat-interface balance of this equation of state reproduces."""
    nx = 64
    x = np.arange(nx)
    l0, g0 = _mechanical_stability(G)
    prof = g0 + (l0 - g0) * 0.5 * (np.tanh((x - 16) / 2.0) - np.tanh((x - 48) / 2.0))
    s = _sim(orc, model=orc.SC_MP, nx=nx, ny=1, nz=1, G=G, rho0_psi=1.0, tau_r=1.0)
    s.init(prof * 1.02)
    s.step(15000)
    r, _, _, t = s.moments()
    liq, gas = r[32], r[0]
    print("SC coexistence G=%g: liquid %.5f gas %.5f (theory %.5f %.5f)" % (G, liq, gas, l0, g0))
    assert abs(liq - l0) / l0 < 2e-3
    assert abs(gas - g0) / g0 < 5e-3
    assert t[6] < 1e-6


def test_sc_two_component_demixing_balance(orc):
    """Two-component SC (cross force of Eq. doublebeltrepulsionforce2, G = 0.9,
    rho_0 = 0.577, so G_eff = G/rho_0^2 = 2.7): with sum_i w_i c_i c_i = I/3 the force is
    -rho_s grad(G_eff c_s^2 rho_s'), so each species has chemical potential
    c_s^2 (ln rho_s + G_eff rho_s').  A flat interface between symmetric phases (a, b) and
    (b, a) then settles where ln(a/b) = G_eff (a - b).  The lattice stencil's higher-order
    terms shift the discrete balance slightly (measured 0.0827 vs 0.0871 mean field), so the
    bound is 6e-3 absolute; a missing 1/rho_0^2 or a sign error moves it by far more."""
    from scipy.optimize import brentq
    nx = 64
    x = np.arange(nx)
    ins = (x >= 16) & (x < 48)
    rr = np.where(ins, 1.0, 0.02)
    rb = np.where(ins, 0.02, 1.0)
    g_eff = 0.9 / 0.577 ** 2
    s = _sim(orc, model=orc.SC_2C, nx=nx, ny=1, nz=1, G=0.9, rho0_psi=0.577)
    s.init(rr, rb)
    s.step(9000)
    r, b, _, _ = s.moments()
    a_, b_ = r[32], b[32]
    tot = a_ + b_
    m = brentq(lambda m: np.log((1 + m) / (1 - m)) - g_eff * tot * m, 1e-6, 1 - 1e-12)
    want_minority = (1 - m) / 2
    print("SC 2C minority fraction %.5f (mean field %.5f)" % (b_ / tot, want_minority))
    assert abs(b_ / tot - want_minority) < 6e-3
    assert abs(r[0] / (r[0] + b[0]) - want_minority) < 6e-3


# ---------------------------------------------------------------- CG repulsion force

def _rep_sim(orc, rr, rb, n):
    s = _sim(orc, nx=n, ny=4, nz=4, rho_r0=1.0, rho_b0=1.0, A=5e-3, rep_pi=0.01, rep_chi=2.0,
             grad_eps=1e-9)
    s.init(rr, rb)
    return s


def test_repulsion_only_at_colour_extrema(orc):
    """A slab on a periodic box has two interfaces; the normals point at each other across
    a link only at the rho^N extrema halfway between them (slab centre x = 15.5, blue
    centre x = 31.5), so F_rep vanishes at every other node.  There the interfaces are
    8 nodes away and psi_rep = (1 - |rho^N|)^2 makes the force negligible against the thin
    film below."""
    n = 32
    ins = inputs.slab(n, 4, 4, 8, 24)
    rr, rb = inputs.two_fluid(ins, 1.0, 1.0)
    s = _rep_sim(orc, rr, rb, n)
    s.step(20)
    F = s.force()[0].reshape(4, 4, n)[0, 0]
    nzx = set(np.nonzero(F)[0].tolist())
    assert nzx <= {14, 15, 16, 17, 30, 31, 0, 1}
    assert np.max(np.abs(F)) < 1e-8


def test_repulsion_in_thin_film(orc):
    """Two red slabs separated by a 4-node blue film centred at x = 20.5 (mirror-symmetric
    box): the two film nodes next to the rho^N minimum have opposite normals across their
    link, so F_rep acts there only, equal and opposite, pointing away from the film centre
    toward the interfaces (outward, Sec. 2.3: it raises the pressure against the
    interfaces and pushes them apart); its total is zero."""
    n = 41
    x = np.arange(n)
    film = (x >= 19) & (x < 23)
    red = ~film & (np.abs(x - 20.5) < 14)
    ins = np.broadcast_to(red[None, None, :], (4, 4, n)).reshape(-1)
    rr, rb = inputs.two_fluid(ins, 1.0, 1.0)
    s = _rep_sim(orc, rr, rb, n)
    s.step(3)
    F = s.force()[0].reshape(4, 4, n)[0, 0]
    nzx = np.nonzero(F)[0]
    assert set(nzx.tolist()) == {20, 21}
    assert F[20] < -1e-4 and abs(F[20] + F[21]) < 1e-15
    Fall = s.force()
    assert np.max(np.abs(Fall[1:])) == 0.0


@pytest.mark.slow
def test_droplet_oscillation_miller_scriven(orc):
    """Sec. 3.2: an ellipsoidal CG droplet (ratio 1, tau = 0.52, A = 0.02, semi-axes
    8.8 / 7.63 / 7.63 in a 28^3 box) oscillates in its second mode at the frequency of
    Eqs. millscriv, millscriv2, millscriv3.  R(t) is the radius along y through the centre
    (rho^N = 0, linearly interpolated), fitted with R_D + a exp(-b t) sin(d t + c); the
    formula takes the run's own R_D and its measured surface tension sigma = dP R_D / 2
    (dP from the CG pressure p = sum_k rho_k (1 - alpha_k)/2 inside and outside, Eq.
    CGpressure), rho_in = rho_out = 1 and nu = (tau - 1/2)/3.  The paper reports 11.5% at
    R_D = 11.65 (Table dropOsc); at R_D ~ 7.6 this run measures 9.5%, held to 10%, and the oscillation must
    decay.  A wrong inertia, viscosity or pressure law moves the frequency by far more."""
    from scipy.optimize import curve_fit
    n, tau, A, a = 28, 0.52, 0.02, 8.8
    b = np.sqrt(512.0 / a)
    c = n // 2
    x, y, z = inputs.grid(n, n, n)
    ins = ((x - c) / a) ** 2 + ((y - c) / b) ** 2 + ((z - c) / b) ** 2 <= 1.0
    rr, rb = inputs.two_fluid(ins, 1.0, 1.0, 0.0, 1)
    s = _sim(orc, lattice=orc.D3Q19, model=orc.CG, nx=n, ny=n, nz=n, rho_r0=1.0, rho_b0=1.0, tau_r=tau,
             tau_b=tau, A=A)
    s.init(rr, rb)

    def radius():
        r, bl, _, _ = s.moments()
        rn = ((r - bl) / (r + bl)).reshape(n, n, n)[c, :, c]  # along y at x = z = centre
        out = []
        for sgn in (1, -1):
            for k in range(c - 1):
                y0, y1 = c + sgn * k, c + sgn * (k + 1)
                if rn[y0] > 0 >= rn[y1]:
                    out.append(k + rn[y0] / (rn[y0] - rn[y1]))
                    break
        assert len(out) == 2
        return np.mean(out)

    ts, rs = [], []
    for t in range(0, 1500, 5):
        ts.append(t)
        rs.append(radius())
        s.step(5)
    ts, rs = np.array(ts, dtype=float), np.array(rs)
    r, bl, _, tot = s.moments()
    rho = (r + bl).reshape(n, n, n)
    dP = 0.4 * (rho[c, c, c] - rho[0, 0, 0])          # alpha_R = alpha_B = 0.2
    RD = rs[-40:].mean()
    sigma = dP * RD / 2
    nu = (tau - 0.5) / 3
    w_star = np.sqrt(24 * sigma / (RD ** 3 * (2 + 3)))                               # Eq. millscriv2
    alpha = 25 * nu / (np.sqrt(2) * RD * (2 + 3) * (2 * np.sqrt(nu)))               # Eq. millscriv3
    w2 = w_star - 0.5 * alpha * np.sqrt(w_star) + 0.25 * alpha ** 2                 # Eq. millscriv
    fit = lambda t, R, amp, damp, d, ph: R + amp * np.exp(-damp * t) * np.sin(d * t + ph)
    sel = ts >= 40
    p, _ = curve_fit(fit, ts[sel], rs[sel], p0=[RD, -0.5, 1e-3, w2, 0.0], maxfev=20000)
    err = (p[3] - w2) / w2
    print(f"Miller-Scriven: R_D {RD:.3f}, sigma {sigma:.5f} (theory {4 / 9 * A * tau:.5f}), "
          f"omega_2 fit {p[3]:.5f} vs formula {w2:.5f} ({err:+.3f}), damping {p[2]:.2e}")
    assert abs(err) < 0.10   # measured -0.095 (deterministic: FP64, per-node work only)
    assert p[2] > 0
    assert 0.8 < sigma / (4 / 9 * A * tau) < 1.1   # sigma = (4/9) A / omega_eff within the Laplace error


def test_repulsion_sign_keeps_colliding_drops_apart(orc):
    """The sign of the repulsion force against the physics the text states for it (Sec. 2.3:
    the force acts outward, repulsive, to keep interfaces apart), on the oracle alone: two
    drops of radius 6 meet head-on at +-0.05 (A = 0.02, tau = 0.6, chi = 2).  Without the
    force they coalesce within 100 steps (red density ~1 on the axis at the contact plane);
    with Pi = 0.03 they stay apart (a blue film remains: red density ~0.14 there after 200
    steps); with the sign reversed (the printed sum of Eq. repForce taken as the force) they
    coalesce as without it, slightly faster at first.  A reversed sign in F_rep fails the
    first or the last assertion."""
    nx, ny, nz = 44, 22, 22
    x, y, z = inputs.grid(nx, ny, nz)
    R = 6.0
    c1, c2 = nx / 2 - R - 1.5, nx / 2 + R + 1.5
    d1 = (x - c1) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2 <= R ** 2
    d2 = (x - c2) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2 <= R ** 2
    rr, rb = inputs.two_fluid(d1 | d2, 1.0, 1.0, 0.0, 1)
    u = np.zeros((3, nx * ny * nz))
    u[0] = np.where(d1, 0.05, np.where(d2, -0.05, 0.0))
    contact = ((x == nx // 2) | (x == nx // 2 - 1)) & (np.abs(y - ny / 2) < 1.5) & (np.abs(z - nz / 2) < 1.5)
    red = {}
    for pi in (0.0, 0.03, -0.03):
        s = _sim(orc, lattice=orc.D3Q19, model=orc.CG, nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1.0, tau_r=0.6,
                 tau_b=0.6, A=0.02, rep_pi=pi, rep_chi=2.0, grad_eps=1e-6)
        s.init(rr, rb, u)
        s.step(50)
        early = float(s.moments()[0][contact].mean())
        s.step(150)
        red[pi] = (early, float(s.moments()[0][contact].mean()))
    print("red density at the contact plane (step 50, step 200):", red)
    assert red[0.03][1] < 0.3                      # repulsive: the drops stay apart
    assert red[0.0][1] > 0.8 and red[-0.03][1] > 0.8  # coalesced without the force and with it reversed
    assert red[-0.03][0] >= red[0.0][0]            # the reversed force pulls the interfaces together
