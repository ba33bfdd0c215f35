"""Seeded synthetic inputs for the two-component LBM workloads.

Geometry and noise only: this module holds none of the method's arithmetic, so both the
CUDA path and the CPU oracle can take their initial fields from it.  Every field is FP64,
node-ordered with x fastest (node = x + nx*(y + ny*z)).

Noise comes from splitmix64(seed, node) (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), mapped to a uniform double in [-1, 1).
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """splitmix64 output for state = seed*golden + (idx+1)*golden, vectorised."""
    with np.errstate(over="ignore"):
        g = np.uint64(0x9E3779B97F4A7C15)
        z = (np.uint64(seed) * g + (idx.astype(np.uint64) + np.uint64(1)) * g) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n doubles uniform in [-1, 1) from splitmix64; ``stream`` separates independent draws."""
    idx = np.arange(n, dtype=np.uint64) + np.uint64(stream) * np.uint64(n)
    bits = splitmix64(seed, idx) >> np.uint64(11)
    return bits.astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


def grid(nx: int, ny: int, nz: int):
    """Node-ordered coordinate arrays (x, y, z), each [N] float64."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.reshape(-1).astype(np.float64), y.reshape(-1).astype(np.float64), \
        z.reshape(-1).astype(np.float64)


def two_fluid(inside: np.ndarray, rho_in: float, rho_out: float, noise: float = 0.0,
              seed: int = 0):
    """Sharp-interface split: component R = rho_in inside, 0 outside; component B the
    complement with rho_out.  ``noise`` scales each density by (1 + noise*U(-1,1))."""
    n = inside.size
    rr = np.where(inside, rho_in, 0.0)
    rb = np.where(inside, 0.0, rho_out)
    if noise:
        rr = rr * (1.0 + noise * uniform_pm1(seed, n, 0))
        rb = rb * (1.0 + noise * uniform_pm1(seed, n, 1))
    return rr, rb


def ellipsoid(nx, ny, nz, semi=(24.0, 20.0, 20.0), centre=None):
    """Indicator of an axis-aligned ellipsoid (2D: ellipse when nz == 1)."""
    x, y, z = grid(nx, ny, nz)
    if centre is None:
        centre = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    cx, cy, cz = centre
    r = ((x - cx) / semi[0]) ** 2 + ((y - cy) / semi[1]) ** 2
    if nz > 1:
        r = r + ((z - cz) / semi[2]) ** 2
    return r <= 1.0


def sphere(nx, ny, nz, radius, centre=None):
    return ellipsoid(nx, ny, nz, (radius, radius, radius), centre)


def jet(nx, ny, nz, radius=10.0, amplitude=1.0, wavelength=None):
    """Cylinder along z, axis at the x-y centre, radius r(z) = R + a cos(2 pi z / lambda).
    The default wavelength nz/round(nz/(4.5 D)) keeps the perturbation periodic."""
    x, y, z = grid(nx, ny, nz)
    if wavelength is None:
        waves = max(1, round(nz / (4.5 * 2.0 * radius)))
        wavelength = nz / waves
    r = radius + amplitude * np.cos(2.0 * np.pi * z / wavelength)
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    return (x - cx) ** 2 + (y - cy) ** 2 <= r ** 2


def capsule(nx, ny, nz, radius=8.0, length=None):
    """Ligament along z: cylinder of ``radius`` and total ``length`` with hemispherical caps."""
    x, y, z = grid(nx, ny, nz)
    if length is None:
        length = 40.0 * 2.0 * radius
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    half = length / 2.0 - radius
    dz = np.clip(np.abs(z - cz) - half, 0.0, None)
    return (x - cx) ** 2 + (y - cy) ** 2 + dz ** 2 <= radius ** 2


def capsule_distance(nx, ny, nz, radius=8.0, length=None):
    """Signed distance to the surface of ``capsule`` (negative inside)."""
    x, y, z = grid(nx, ny, nz)
    if length is None:
        length = 40.0 * 2.0 * radius
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    half = length / 2.0 - radius
    dz = np.clip(np.abs(z - cz) - half, 0.0, None)
    return np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + dz ** 2) - radius


def diffuse_two_fluid(distance: np.ndarray, rho_in: float, rho_out: float, width: float,
                      noise: float = 0.0, seed: int = 0):
    """Interface of finite width instead of a step: component R = rho_in (1 - tanh(d/w))/2,
    component B = rho_out (1 + tanh(d/w))/2 at signed distance d (negative inside);
    ``noise`` as in two_fluid."""
    n = distance.size
    t = np.tanh(distance / width)
    rr = rho_in * 0.5 * (1.0 - t)
    rb = rho_out * 0.5 * (1.0 + t)
    if noise:
        rr = rr * (1.0 + noise * uniform_pm1(seed, n, 0))
        rb = rb * (1.0 + noise * uniform_pm1(seed, n, 1))
    return rr, rb


def slab(nx, ny, nz, lo, hi, axis=0):
    """Indicator lo <= coordinate < hi along ``axis`` (flat interfaces, layered flows)."""
    c = grid(nx, ny, nz)[axis]
    return (c >= lo) & (c < hi)


def emulsion(nx, ny, nz, count=200, r_mean=10.0, r_spread=2.0, gap=3.0, seed=4, max_tries=200000):
    """Random sequential addition of non-overlapping spheres (periodic distances), radii
    uniform in [r_mean - r_spread, r_mean + r_spread], at least ``gap`` nodes apart.
    Returns (indicator, list of (cx, cy, cz, r))."""
    rng_vals = uniform_pm1(seed, 4 * max_tries, 7).reshape(max_tries, 4)
    L = np.array([nx, ny, nz], dtype=np.float64)
    placed = []
    for t in range(max_tries):
        if len(placed) >= count:
            break
        u = rng_vals[t]
        c = (u[:3] + 1.0) * 0.5 * L
        r = r_mean + r_spread * u[3]
        ok = True
        for (px, py, pz, pr) in placed:
            d = np.abs(c - np.array([px, py, pz]))
            d = np.minimum(d, L - d)
            if np.sqrt((d * d).sum()) < r + pr + gap:
                ok = False
                break
        if ok:
            placed.append((c[0], c[1], c[2], r))
    inside = np.zeros((nz, ny, nx), dtype=bool)
    for (px, py, pz, pr) in placed:
        # the sphere's bounding box, wrapped periodically
        ix = np.arange(int(np.floor(px - pr)), int(np.ceil(px + pr)) + 1)
        iy = np.arange(int(np.floor(py - pr)), int(np.ceil(py + pr)) + 1)
        iz = np.arange(int(np.floor(pz - pr)), int(np.ceil(pz + pr)) + 1)
        dz, dy, dx = np.meshgrid(iz - pz, iy - py, ix - px, indexing="ij")
        box = dx * dx + dy * dy + dz * dz <= pr * pr
        sub = np.ix_(iz % nz, iy % ny, ix % nx)
        inside[sub] |= box
    return inside.reshape(-1), placed


def channel_walls(nx, ny, nz):
    """Solid mask with walls on the planes y = 0 and y = ny-1 (uint8, 1 = solid)."""
    _, y, _ = grid(nx, ny, nz)
    return ((y == 0) | (y == ny - 1)).astype(np.uint8)


def shear_wave_velocity(nx, ny, nz, amplitude=1e-3):
    """u_x(y) = U sin(2 pi y / ny), u_y = u_z = 0, as a [3, N] array."""
    _, y, _ = grid(nx, ny, nz)
    u = np.zeros((3, y.size))
    u[0] = amplitude * np.sin(2.0 * np.pi * y / ny)
    return u
