"""Brute-force NumPy transcription of one lattice Boltzmann step, written from the paper
independently of the C oracle, to pin the oracle on tiny lattices (8 x 8 D2Q9, 4 x 4 x 4
D3Q19).  Whole-lattice array operations: shifts by np.roll, no per-node loops, no code or
table shared with oracle/ or the CUDA library.

Passages: SC Sec. 2.1 (Eqs. interactionforceMP, pseudopotential, guoforce2, source,
collisSC, equiliSC, streamingSC; two-component cross force Eq. doublebeltrepulsionforce2);
CG Sec. 2.2 (Eqs. density, totalMomentum2, interpVisc, effRelax, equiliCG, phi, tensorG,
gamma, BGK, perturbationOp, recoloringOpR/B, cosphi, streamingCG) with forces by Guo
(Eqs. guoforce, source); CG repulsion force Sec. 2.3 (Eqs. repForce, potential, normal1,
normal2).  The readings where the paper is silent or garbled are the ones the library
documents: perturbation A|grad rho^N|[...] on the total population, phi_i^k in the BGK
equilibrium, one omega_eff for both colours with nu_k = (tau_k - 1/2)/3, isotropic
gradients 3 sum_i w_i phi(x + c_i) c_i as opposite-pair differences with a wall
neighbour's value replaced by the centre's, Guo forcing on the total post-BGK population,
halfway bounce-back, psi_rep = (1 -+ |rho^N|)^chi with H(0) = 0 and undefined normals
(|grad rho^N| <= eps) contributing nothing, barycentric velocity for two-component SC.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# ---- velocity sets: rest, then opposite pairs (2p+1, 2p+2) ----
_D2Q9 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0)]
_D3Q19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
          (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
          (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


class Lattice:
    def __init__(self, d3: bool):
        self.c = np.array(_D3Q19 if d3 else _D2Q9, dtype=np.int64)
        self.q = len(self.c)
        c2 = (self.c ** 2).sum(axis=1)
        self.group = np.where(c2 == 0, 0, np.where(c2 == 1, 1, 2))
        if d3:
            # Eq. weights; B_i, psi_i, xi_i as printed with Eqs. perturbationOp, equiliCG
            w, B, psi, xi = (1 / 3, 1 / 18, 1 / 36), (-2 / 9, 1 / 54, 1 / 27), (-5 / 2, -1 / 6, 1 / 24), (0, 1 / 4, 1 / 8)
            self.phi_split = (1 / 12, 1 / 24)      # Eq. phi: (1 - alpha)/12, (1 - alpha)/24
        else:
            # D2Q9 analogues (chosen to satisfy the same moment identities)
            w, B, psi, xi = (4 / 9, 1 / 9, 1 / 36), (-4 / 27, 2 / 27, 5 / 108), (-8 / 3, -1 / 6, 1 / 12), (0, 1 / 2, 1 / 8)
            self.phi_split = (1 / 5, 1 / 20)
        pick = lambda t: np.array([t[g] for g in self.group], dtype=np.float64)
        self.w, self.B, self.psi, self.xi = pick(w), pick(B), pick(psi), pick(xi)
        self.norm = np.sqrt(c2.astype(np.float64))
        self.opp = np.array([np.flatnonzero((self.c == -ci).all(axis=1))[0] for ci in self.c])

    def phi(self, alpha):
        return np.array([alpha if g == 0 else (1 - alpha) * self.phi_split[g - 1] for g in self.group])


def shift(a, c):
    """a(x + c) on the periodic lattice; arrays are indexed [..., z, y, x]."""
    return np.roll(a, shift=(-int(c[2]), -int(c[1]), -int(c[0])), axis=(-3, -2, -1))


def unshift(a, c):
    """value at x - c moved to x, i.e. the push of a along c."""
    return np.roll(a, shift=(int(c[2]), int(c[1]), int(c[0])), axis=(-3, -2, -1))


@dataclass
class Params:
    d3: bool
    model: str                 # "cg", "sc_mp", "sc_2c", "sc_mr"
    shape: tuple               # (nz, ny, nx)
    rho_r0: float = 1.0
    rho_b0: float = 1.0
    alpha_b: float = 0.2
    tau_r: float = 1.0
    tau_b: float = 1.0
    A: float = 0.0
    beta: float = 0.7
    enhanced: bool = True
    color_norm: bool = False
    rep_pi: float = 0.0
    rep_chi: float = 2.0
    rep_printed: bool = False  # psi_rep = (1 + |rho^N|)^chi as printed
    grad_eps: float = 0.0
    G: float = 0.0
    rho0: float = 1.0
    body: tuple = (0.0, 0.0, 0.0)
    Ga: tuple = (0.0, 0.0)     # sc_mr: attractive self-couplings (belt 1, weights w)
    Gr: tuple = (0.0, 0.0)     # sc_mr: repulsive self-couplings (belts 1 + 2, weights p)
    solid: np.ndarray | None = None


# Eq. pweights: the forcing weight of a belt vector depends on |c|^2 only
P_OF_R2 = {1: 4 / 135, 2: 1 / 63, 3: 2 / 315, 4: 5 / 1512, 5: 1 / 945, 6: 1 / 1890, 8: 1 / 15120}


def belt_vectors():
    """Non-zero integer vectors of belts 1 and 2 (|c|^2 <= 8) with their weights p."""
    r = np.arange(-2, 3)
    out = []
    for x in r:
        for y in r:
            for z in r:
                r2 = int(x * x + y * y + z * z)
                if r2 in P_OF_R2:
                    out.append(((int(x), int(y), int(z)), P_OF_R2[r2]))
    return out


class BruteForce:
    def __init__(self, p: Params):
        self.p = p
        self.L = Lattice(p.d3)
        self.solid = np.zeros(p.shape, bool) if p.solid is None else p.solid.astype(bool).reshape(p.shape)
        self.fluid = ~self.solid
        # Eq. gamma: rho_R0 / rho_B0 = (1 - alpha_B) / (1 - alpha_R)
        self.alpha_r = 1 - (1 - p.alpha_b) * p.rho_b0 / p.rho_r0
        self.phis = (self.L.phi(self.alpha_r), self.L.phi(p.alpha_b))
        self.K = 1 if p.model == "sc_mp" else 2
        self.f = None

    # ---- fields ----
    def grad(self, s):
        """3 sum_i w_i s(x + c_i) c_i as pair differences; solid neighbours give s(x)."""
        g = np.zeros((3,) + s.shape)
        L = self.L
        for i in range(1, L.q, 2):
            sp = np.where(shift(self.solid, L.c[i]), s, shift(s, L.c[i]))
            sm = np.where(shift(self.solid, -L.c[i]), s, shift(s, -L.c[i]))
            for a in range(3):
                if L.c[i][a]:
                    g[a] += 3 * L.w[i] * (sp - sm) * L.c[i][a]
        return g

    def colour(self, rr, rb):
        if self.p.color_norm:
            rr, rb = rr / self.p.rho_r0, rb / self.p.rho_b0
        return (rr - rb) / (rr + rb)

    def rep_force(self, rhoN, gN):
        p, L = self.p, self.L
        gabs = np.sqrt((gN ** 2).sum(axis=0))
        ok = gabs > p.grad_eps
        n = np.where(ok, gN / np.where(ok, gabs, 1.0), 0.0)
        acc = np.zeros_like(gN)
        for i in range(1, L.q):
            ci = L.c[i].astype(np.float64)
            n2 = shift(n, L.c[i])
            ok2 = shift(ok, L.c[i]) & ~shift(self.solid, L.c[i])
            nc = np.tensordot(ci, n, axes=(0, 0))
            n2c = np.tensordot(ci, n2, axes=(0, 0))
            H = (-(nc * n2c) > 0) & ok2
            acc += np.where(H, (nc * n + n2c * n2) / L.norm[i], 0.0)
        base = 1 + np.abs(rhoN) if p.rep_printed else 1 - np.abs(rhoN)
        F = -p.rep_pi * base ** p.rep_chi * acc   # outward: away from the rho^N extremum
        return np.where(ok & self.fluid, F, 0.0)

    # ---- equilibria and operators ----
    def cg_feq(self, k, rho_k, u, g_k, nubar):
        L, p = self.L, self.p
        uu = (u ** 2).sum(axis=0)
        ug = (u * g_k).sum(axis=0)
        out = np.empty((L.q,) + rho_k.shape)
        for i in range(L.q):
            ci = L.c[i].astype(np.float64)
            cu = np.tensordot(ci, u, axes=(0, 0))
            cg = np.tensordot(ci, g_k, axes=(0, 0))
            enh = nubar * (L.psi[i] * ug + L.xi[i] * 2 * cu * cg) if p.enhanced else 0.0
            out[i] = enh + rho_k * (self.phis[k][i] + L.w[i] * (3 * cu + 4.5 * cu * cu - 1.5 * uu))
        return out

    def sc_feq(self, rho, u):
        L = self.L
        uu = (u ** 2).sum(axis=0)
        out = np.empty((L.q,) + rho.shape)
        for i in range(L.q):
            cu = np.tensordot(L.c[i].astype(np.float64), u, axes=(0, 0))
            out[i] = rho * L.w[i] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
        return out

    def guo(self, u, F, omega):
        L = self.L
        uF = (u * F).sum(axis=0)
        out = np.empty((L.q,) + u.shape[1:])
        for i in range(L.q):
            ci = L.c[i].astype(np.float64)
            cu = np.tensordot(ci, u, axes=(0, 0))
            cF = np.tensordot(ci, F, axes=(0, 0))
            out[i] = L.w[i] * (1 - 0.5 * omega) * (3 * (cF - uF) + 9 * cu * cF)
        return out

    def body_field(self):
        return np.broadcast_to(np.array(self.p.body, dtype=np.float64).reshape(3, 1, 1, 1),
                               (3,) + self.p.shape).copy()

    def viscosity(self, rr, rb):
        nu_r, nu_b = (self.p.tau_r - 0.5) / 3, (self.p.tau_b - 0.5) / 3
        rho = rr + rb
        nubar = 1 / ((rr / rho) / nu_r + (rb / rho) / nu_b)
        return nubar, 2 / (6 * nubar + 1)

    def momentum(self, f):
        return np.tensordot(self.L.c.T.astype(np.float64), f.sum(axis=0), axes=(1, 0))

    # ---- init / step ----
    def init(self, rho_r, rho_b=None, u=None):
        with np.errstate(divide="ignore", invalid="ignore"):  # 0/0 on wall nodes, masked out
            return self._init(rho_r, rho_b, u)

    def _init(self, rho_r, rho_b, u):
        p, L = self.p, self.L
        rr = rho_r.reshape(p.shape).astype(np.float64)
        rb = np.zeros(p.shape) if rho_b is None else rho_b.reshape(p.shape).astype(np.float64)
        u = np.zeros((3,) + p.shape) if u is None else u.reshape((3,) + p.shape)
        f = np.zeros((self.K, L.q) + p.shape)
        if p.model == "cg":
            nubar, _ = self.viscosity(rr, rb)
            f[0] = self.cg_feq(0, rr, u, self.grad(rr), nubar)
            f[1] = self.cg_feq(1, rb, u, self.grad(rb), nubar)
        else:
            f[0] = self.sc_feq(rr, u)
            if self.K == 2:
                f[1] = self.sc_feq(rb, u)
        self.f = np.where(self.fluid, f, 0.0)
        return self

    def stream(self, post):
        L = self.L
        post = np.where(self.fluid, post, 0.0)
        new = np.zeros_like(post)
        for i in range(L.q):
            blocked = shift(self.solid, L.c[i])  # x + c_i is a wall
            new[:, i] += unshift(np.where(blocked, 0.0, post[:, i]), L.c[i])
            new[:, L.opp[i]] += np.where(blocked, post[:, i], 0.0)
        return np.where(self.fluid, new, 0.0)

    def step(self, n=1):
        with np.errstate(divide="ignore", invalid="ignore"):  # 0/0 on wall nodes, masked out
            for _ in range(n):
                self.f = self.stream(self.cg_post() if self.p.model == "cg" else self.sc_post())
        return self

    def cg_post(self):
        p, L, f = self.p, self.L, self.f
        rr, rb = f[0].sum(axis=0), f[1].sum(axis=0)
        rho = rr + rb
        rhoN = self.colour(rr, rb)
        gN, gR, gB = self.grad(rhoN), self.grad(rr), self.grad(rb)
        F = self.body_field()
        if p.rep_pi != 0.0:
            F = F + self.rep_force(rhoN, gN)
        u = (self.momentum(f) + 0.5 * F) / rho
        nubar, omega = self.viscosity(rr, rb)
        fstar = (f[0] - omega * (f[0] - self.cg_feq(0, rr, u, gR, nubar))
                 + f[1] - omega * (f[1] - self.cg_feq(1, rb, u, gB, nubar)))
        fstar = fstar + self.guo(u, F, omega)
        gabs = np.sqrt((gN ** 2).sum(axis=0))
        has = gabs > p.grad_eps
        safe = np.where(has, gabs, 1.0)
        post = np.empty_like(f)
        beta_term = p.beta * rr * rb / rho ** 2
        for i in range(L.q):
            cg = np.tensordot(L.c[i].astype(np.float64), gN, axes=(0, 0))
            pert = np.where(has, p.A * gabs * (L.w[i] * cg * cg / safe ** 2 - L.B[i]), 0.0)
            fs = fstar[i] + pert
            cosphi = np.where(has, cg / (L.norm[i] * safe), 0.0) if i else 0.0
            feq0 = rr * self.phis[0][i] + rb * self.phis[1][i]
            post[0, i] = rr / rho * fs + beta_term * cosphi * feq0
            post[1, i] = fs - post[0, i]
        return post

    def _weighted_sum(self, s, vectors):
        """sum_j wt_j s(x + c_j) c_j over (c, wt) pairs; a solid neighbour gives s(x)."""
        acc = np.zeros((3,) + s.shape)
        for c, wt in vectors:
            v = np.where(shift(self.solid, c), s, shift(s, c))
            for a in range(3):
                if c[a]:
                    acc[a] += wt * v * c[a]
        return acc

    def sc_post(self):
        p, L, f = self.p, self.L, self.f
        rhos = [f[k].sum(axis=0) for k in range(self.K)]
        body = self.body_field()
        if p.model == "sc_mr":
            # Eq. benziforces: attractive belt 1 (w), repulsive belts 1+2 (p), cross (w)
            lattice = [(L.c[i], L.w[i]) for i in range(1, L.q)]
            belts = belt_vectors()
            rho = rhos[0] + rhos[1]
            Fs = []
            for k in range(2):
                Psi = p.rho0 * (1 - np.exp(-rhos[k] / p.rho0))
                Fa = -p.Ga[k] * Psi * self._weighted_sum(Psi, lattice)
                Fr = -p.Gr[k] * Psi * self._weighted_sum(Psi, belts)
                Fx = -(p.G / p.rho0 ** 2) * rhos[k] * self._weighted_sum(rhos[1 - k], lattice)
                Fs.append(Fa + Fr + Fx + body * rhos[k] / rho)
            u = (self.momentum(f) + 0.5 * sum(Fs)) / rho
            post = np.empty_like(f)
            for k, tau in enumerate((p.tau_r, p.tau_b)):
                post[k] = f[k] - (f[k] - self.sc_feq(rhos[k], u)) / tau + self.guo(u, Fs[k], 1 / tau)
            return post
        if p.model == "sc_mp":
            rho = rhos[0]
            psi = p.rho0 * (1 - np.exp(-rho / p.rho0))
            s = np.zeros((3,) + p.shape)
            for i in range(1, L.q):
                v = np.where(shift(self.solid, L.c[i]), psi, shift(psi, L.c[i]))
                for a in range(3):
                    s[a] += L.w[i] * v * L.c[i][a]
            Fs = [-p.G * psi * s + body]
        else:
            geff = p.G / p.rho0 ** 2
            rho = rhos[0] + rhos[1]
            Fs = []
            for k in range(2):
                other = rhos[1 - k]
                s = np.zeros((3,) + p.shape)
                for i in range(1, L.q):
                    v = np.where(shift(self.solid, L.c[i]), other, shift(other, L.c[i]))
                    for a in range(3):
                        s[a] += L.w[i] * v * L.c[i][a]
                Fs.append(-geff * rhos[k] * s + body * rhos[k] / rho)
        u = (self.momentum(f) + 0.5 * sum(Fs)) / rho
        taus = (p.tau_r, p.tau_b)
        post = np.empty_like(f)
        for k in range(self.K):
            feq = self.sc_feq(rhos[k], u)
            post[k] = f[k] - (f[k] - feq) / taus[k] + self.guo(u, Fs[k], 1 / taus[k])
        return post

    def pops(self):
        """[K][Q][N] in node order x + nx (y + ny z)."""
        return self.f.reshape(self.K, self.L.q, -1)
