"""Host-side measurements of the paper's benchmark observables, from FP64 moments (the
GPU's lbm_moments or the oracle's): the Laplace pressure jump (Sec. 3.1, Eqs.
YoungLaplace, rhoin, rhoout), the droplet radius along an axis and its oscillation
frequency (Sec. 3.2), and the droplets of a broken jet with their masses (Sec. 3.4).
Measurement code only: it reads densities and computes no part of the step."""
from __future__ import annotations

import numpy as np


def colour(rho_r, rho_b):
    return (rho_r - rho_b) / (rho_r + rho_b)


def eps_level(col) -> float:
    """Eqs. rhoin / rhoout: eps = 1 - 0.1^n with the largest n <= 10 such that both
    phases still have a node beyond +-eps."""
    for k in range(10, 0, -1):
        e = 1 - 0.1 ** k
        if (col >= e).any() and (col <= -e).any():
            return e
    return 0.0


def pressure_jump(rho_r, rho_b, cs2_r: float, cs2_b: float, eps: float | None = None) -> float:
    """p_in - p_out with p = sum_k c_{s,k}^2 rho_k (Eq. CGpressure), the bulk densities
    taken as the means over the nodes beyond +-eps (Eqs. rhoin, rhoout); eps = None takes
    the field's own level (eps_level)."""
    col = colour(rho_r, rho_b)
    e = eps_level(col) if eps is None else eps
    inside, outside = col >= e, col <= -e
    p = cs2_r * rho_r + cs2_b * rho_b
    return float(p[inside].mean() - p[outside].mean())


def radius_along_x(rho_r, rho_b, shape) -> float:
    """Half the distance between the two rho^N = 0 crossings on the x line through the box
    centre (linear interpolation between nodes); shape = (nz, ny, nx)."""
    nz, ny, nx = shape
    col = colour(rho_r, rho_b).reshape(shape)
    line = col[nz // 2, ny // 2, :] if nz > 1 else col[0, ny // 2, :]
    pos = line > 0
    idx = np.nonzero(np.diff(pos.astype(np.int8)))[0]
    if len(idx) < 2:
        return float("nan")
    cr = [i + line[i] / (line[i] - line[i + 1]) for i in idx]
    return 0.5 * float(cr[-1] - cr[0])


def endpoint_along_z(rho_r, rho_b, shape) -> float:
    """Position of the upper rho^N = 0 crossing on the z line through the box centre,
    relative to the centre plane (linear interpolation between nodes); shape = (nz, ny, nx)."""
    nz, ny, nx = shape
    col = colour(rho_r, rho_b).reshape(shape)
    line = col[:, ny // 2, nx // 2]
    idx = np.nonzero(np.diff((line > 0).astype(np.int8)))[0]
    if len(idx) == 0:
        return float("nan")
    i = idx[-1]
    return float(i + line[i] / (line[i] - line[i + 1]) - (nz - 1) / 2.0)


def oscillation_frequency(r, dt: float) -> float:
    """Angular frequency of a decaying oscillation r(t) sampled every dt steps, from a
    least-squares fit of c + a exp(-g t) cos(w t + p); the zero crossings of r - mean(r)
    (two per period) give the starting w."""
    from scipy.optimize import curve_fit
    r = np.asarray(r, dtype=float)
    t = np.arange(1, len(r) + 1) * dt
    d = r - r.mean()
    idx = np.nonzero(np.sign(d[:-1]) * np.sign(d[1:]) < 0)[0]
    if len(idx) < 2:
        return float("nan")
    w0 = np.pi / (np.diff(t[idx]).mean())
    model = lambda tt, c, a, g, w, ph: c + a * np.exp(-g * tt) * np.cos(w * tt + ph)
    best = None
    for ph in np.linspace(-np.pi, np.pi, 8, endpoint=False):
        try:
            par, _ = curve_fit(model, t, r, p0=(r.mean(), np.ptp(r) / 2, 1.0 / t[-1], w0, ph), maxfev=20000)
        except RuntimeError:
            continue
        res = np.sum((model(t, *par) - r) ** 2)
        if best is None or res < best[0]:
            best = (res, par)
    return float(abs(best[1][3])) if best is not None else float("nan")


def periodic_components(mask):
    """Connected components (face neighbours) of a boolean field on a periodic box:
    labels >= 1, 0 outside the mask."""
    from scipy import ndimage
    lab, n = ndimage.label(mask)
    parent = np.arange(n + 1)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for ax in range(mask.ndim):
        a = np.take(lab, 0, axis=ax)
        b = np.take(lab, -1, axis=ax)
        both = (a > 0) & (b > 0)
        for u, v in zip(a[both], b[both]):
            ru, rv = find(u), find(v)
            if ru != rv:
                parent[ru] = rv
    roots = np.array([find(i) for i in range(n + 1)])
    return roots[lab]


def droplet_masses(rho_r, rho_b, shape):
    """Red mass of every connected region with rho^N > 0, largest first."""
    lab = periodic_components(colour(rho_r, rho_b).reshape(shape) > 0)
    r = rho_r.reshape(shape)
    ids = np.unique(lab[lab > 0])
    return sorted((float(r[lab == i].sum()) for i in ids), reverse=True)
