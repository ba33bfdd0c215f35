"""Seeded parity cases shared by the GPU tests: each yields the parameters for both sides
and the initial fields from the input generators (geometry and noise only)."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from paper_2110_05197_gb300 import inputs

# SC multiphase coexistence at G = -5 (mechanical stability with Guo forcing)
SC_LIQ, SC_GAS = 1.8884, 0.1194


@dataclass
class Case:
    name: str
    kw: dict                    # shared parameters (oracle.Params / lbm.Params field names)
    rho_r: np.ndarray
    rho_b: np.ndarray | None = None
    u: np.ndarray | None = None
    solid: np.ndarray | None = None


def cg_drop3d(nx=20, ny=18, nz=17, ratio=10.0, seed=2, **extra):
    rr, rb = inputs.two_fluid(inputs.ellipsoid(nx, ny, nz, (7, 6, 5)), 1.0, 1.0 / ratio, 0.01, seed)
    kw = dict(lattice=1, model=0, nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1.0 / ratio, tau_r=1.0, tau_b=0.7,
              A=5e-3)
    kw.update(extra)
    return Case("cg_drop3d", kw, rr, rb)


def cg_drop2d(n=40, seed=1, **extra):
    rr, rb = inputs.two_fluid(inputs.sphere(n, n + 3, 1, 10), 1.0, 1.0, 0.0, seed)
    kw = dict(lattice=0, model=0, nx=n, ny=n + 3, nz=1, rho_r0=1.0, rho_b0=1.0, A=1e-2)
    kw.update(extra)
    return Case("cg_drop2d", kw, rr, rb)


def cg_walls3d(nx=12, ny=14, nz=10, **extra):
    solid = inputs.channel_walls(nx, ny, nz)
    ins = inputs.sphere(nx, ny, nz, 4.0)
    rr, rb = inputs.two_fluid(ins, 1.0, 0.5, 0.01, 5)
    rr = np.where(solid, 0.0, rr)
    rb = np.where(solid, 0.0, rb)
    kw = dict(lattice=1, model=0, nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=0.5, tau_r=0.9, tau_b=0.6, A=4e-3,
              body_force=(1e-5, 0.0, 2e-6))
    kw.update(extra)
    return Case("cg_walls3d", kw, rr, rb, None, solid)


def sc_mp3d(nx=20, ny=18, nz=17, seed=3, **extra):
    ins = inputs.sphere(nx, ny, nz, 5.5)
    rho = np.where(ins, SC_LIQ, SC_GAS) * (1 + 0.01 * inputs.uniform_pm1(seed, nx * ny * nz))
    kw = dict(lattice=1, model=1, nx=nx, ny=ny, nz=nz, G=-5.0, rho0_psi=1.0, tau_r=1.0)
    kw.update(extra)
    return Case("sc_mp3d", kw, rho)


def sc_2c3d(nx=20, ny=18, nz=17, seed=4, **extra):
    rr, rb = inputs.two_fluid(inputs.sphere(nx, ny, nz, 5.5), 1.0, 1.0, 0.01, seed)
    kw = dict(lattice=1, model=2, nx=nx, ny=ny, nz=nz, G=0.9, rho0_psi=0.577, tau_r=1.0, tau_b=0.8)
    kw.update(extra)
    return Case("sc_2c3d", kw, rr + 0.03, rb + 0.03)


def sc_walls2d(nx=24, ny=20, **extra):
    solid = inputs.channel_walls(nx, ny, 1)
    ins = inputs.sphere(nx, ny, 1, 5.0)
    rho = np.where(ins, SC_LIQ, SC_GAS)
    rho = np.where(solid, 0.0, rho)
    kw = dict(lattice=0, model=1, nx=nx, ny=ny, nz=1, G=-5.0, rho0_psi=1.0, tau_r=0.9,
              body_force=(2e-6, 0.0, 0.0))
    kw.update(extra)
    return Case("sc_walls2d", kw, rho, None, None, solid)


def sc_mr3d(nx=14, ny=12, nz=11, seed=7, walls=False, **extra):
    """Multicomponent SC with multirange potentials (Eq. benziforces): a drop of species A
    (1.18 with 0.18 of B, Table dropcolParams set 1) in B, the printed self-couplings
    G^a = (-9, -8), G^r = (8.1, 7.1), rho_0 = 0.83, and the cross coupling G_AB = 1.215
    (three times the printed 0.405, which with these lattice weights does not demix)."""
    n = nx * ny * nz
    ins = inputs.ellipsoid(nx, ny, nz, (4.5, 3.8, 3.4))
    rr = np.where(ins, 1.18, 0.18) * (1 + 0.01 * inputs.uniform_pm1(seed, n, 0))
    rb = np.where(ins, 0.18, 1.18) * (1 + 0.01 * inputs.uniform_pm1(seed, n, 1))
    kw = dict(lattice=1, model=3, nx=nx, ny=ny, nz=nz, Ga=(-9.0, -8.0), Gr=(8.1, 7.1), G=1.215, rho0_psi=0.83,
              tau_r=1.0, tau_b=0.9)
    solid = None
    if walls:
        solid = inputs.channel_walls(nx, ny, nz)
        rr, rb = np.where(solid, 0.0, rr), np.where(solid, 0.0, rb)
        kw["body_force"] = (1e-5, 0.0, 2e-6)
    kw.update(extra)
    return Case("sc_mr3d", kw, rr, rb, None, solid)


def cg_rep3d(nx=30, ny=16, nz=15, seed=6, **extra):
    """Two droplets about two nodes apart, with different radii and offset centres so that
    the normals in the gap are generic (no symmetry puts a Heaviside argument at FP32
    resolution): the CG repulsion force (Eq. repForce) acts in the gap."""
    x, y, z = inputs.grid(nx, ny, nz)
    d1 = (x - 8.5) ** 2 + (y - 7.5) ** 2 + (z - 7) ** 2 <= 5.2 ** 2
    d2 = (x - 19.7) ** 2 + (y - 8.8) ** 2 + (z - 7.9) ** 2 <= 4.6 ** 2
    rr, rb = inputs.two_fluid(d1 | d2, 1.0, 1.0, 0.01, seed)
    kw = dict(lattice=1, model=0, nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1.0, A=5e-3, rep_pi=0.02, rep_chi=2.0,
              grad_eps=1e-7)
    kw.update(extra)
    return Case("cg_rep3d", kw, rr, rb)


def cg_rep_film(nx=41, ny=6, nz=5, **extra):
    """Two red slabs and a 4-node blue film, seeded noise.  At the film centre rho^N has an
    extremum with both colours present, so grad_eps = 1e-4 switches off the recolouring
    direction where |grad rho^N| is below FP32 resolution."""
    x, _, _ = inputs.grid(nx, ny, nz)
    film = (x >= 19) & (x < 23)
    red = ~film & (np.abs(x - 20.5) < 14)
    rr, rb = inputs.two_fluid(red, 1.0, 1.0, 0.01, 8)
    kw = dict(lattice=1, model=0, nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1.0, A=5e-3, rep_pi=0.01, rep_chi=2.0,
              grad_eps=1e-4, rep_psi_kind=0)
    kw.update(extra)
    return Case("cg_rep_film", kw, rr, rb)


SMALL_CASES = {
    "cg_drop3d": cg_drop3d,
    # sizes the TMA-staged kernel takes (nx % 32 == 0, ny % 8 == 0)
    "cg_tma3d": lambda: cg_drop3d(nx=32, ny=16, nz=13),
    "cg_tma_walls": lambda: cg_walls3d(nx=32, ny=16, nz=9),
    "sc_tma3d": lambda: sc_mp3d(nx=32, ny=16, nz=14),
    "sc2c_tma3d": lambda: sc_2c3d(nx=64, ny=24, nz=5),
    "cg_drop2d": cg_drop2d,
    "cg_walls3d": cg_walls3d,
    "cg_std_norm": lambda: cg_drop3d(enhanced_eq=0, color_norm=1, ratio=4.0),
    "sc_mp3d": sc_mp3d,
    "sc_2c3d": sc_2c3d,
    "sc_walls2d": sc_walls2d,
    "sc_mr3d": sc_mr3d,
    "sc_mr_walls": lambda: sc_mr3d(nx=13, ny=12, nz=10, walls=True),
    "cg_rep3d": cg_rep3d,
    "cg_rep_film": cg_rep_film,
    # the printed psi_rep = (1 + |rho^N|)^chi is largest where |grad rho^N| is near zero and
    # the normal is rounding noise (Pi = 0.02 blows up within 90 steps on the oracle); a
    # grad_eps of 1e-3 keeps only well-defined normals
    "cg_rep_walls": lambda: cg_walls3d(rep_pi=0.001, rep_chi=1.5, grad_eps=1e-3, rep_psi_kind=1),
}


def oracle_sim(orc, case: Case, threads: int | None = None):
    if threads:
        orc.set_threads(threads)
    s = orc.OracleSim(orc.Params(**case.kw))
    s.init(case.rho_r, case.rho_b, case.u, case.solid)
    return s


def gpu_lattice(lbm, case: Case, precision: int, **extra):
    import torch
    kw = dict(case.kw)
    kw.update(extra)
    lat = lbm.Lattice(lbm.Params(precision=precision, **kw))
    dev = lat.device

    def t(a, dt=torch.float64):
        return None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)

    lat.init(t(case.rho_r), t(case.rho_b), t(case.u), t(case.solid, torch.uint8))
    return lat


# Lattices for the ring kernel (512-node tiles, 32 x 16 or 64 x 8, clusters of nx / TX).
RING_CASES = {
    "cg_ring32": lambda: cg_drop3d(nx=32, ny=16, nz=13),                   # 32 x 16: cluster of 1
    "cg_ring64": lambda: cg_drop3d(nx=64, ny=32, nz=10),                   # 32 x 16: 2; 64 x 8: 1
    "cg_ring96": lambda: cg_drop3d(nx=96, ny=16, nz=7, ratio=3.0),         # 32 x 16: 3
    "cg_ring_body": lambda: cg_drop3d(nx=32, ny=16, nz=9, body_force=(1e-5, 0.0, 2e-6)),
    "sc_ring64": lambda: sc_mp3d(nx=64, ny=16, nz=14),                     # 32 x 16: 2; 64 x 8: 1
    "cg_ring256": lambda: cg_drop3d(nx=256, ny=16, nz=6),                  # 32 x 16: 8 (the largest cluster)
    "sc_ring512": lambda: sc_mp3d(nx=512, ny=16, nz=14),                   # 64 x 8 and 64 x 4: 8
}


def ring_runs(kw: dict, precision: int, tiling) -> bool:
    """Whether the library runs a tiling on the ring kernel: 32 x 16 and 64 x 8 tiles
    (one block per SM; else it runs 32 x 8 tiles) and 64 x 4 tiles (two blocks per SM;
    else the cluster kernel), for D3Q19, FP32/FP16/BF16 storage, CG or SC multiphase, no
    walls, no repulsion force, two-buffer streaming, nx % TX == ny % TY == 0,
    nx / TX <= 8, and a shared-memory footprint within the block's share: FP32 CG runs
    only 32 x 16 tiles."""
    tx, ty = tiling[0], tiling[1]
    if kw.get("lattice", 1) != 1 or precision == 0 or kw.get("model", 0) not in (0, 1):
        return False
    if kw.get("rep_pi", 0.0) or kw.get("streaming", 0):
        return False
    if kw["nx"] % tx or kw["ny"] % ty or kw["nx"] // tx > 8:
        return False
    return not (kw.get("model", 0) == 0 and precision == 1 and tx == 64)
