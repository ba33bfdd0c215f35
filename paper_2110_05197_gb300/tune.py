"""Launch-shape autotuner for the fused step kernel.

For a lattice it times a handful of tilings (block columns tx x ty, z planes per block tz,
tz = 0 for the persistent grid; 32 x 8 selects the TMA-staged kernel where the lattice
allows it) on the lattice's own
state, keeps the fastest, and restores the state bit for bit (raw state save/load), so
tuning never changes a simulation's result.  The choice is cached per lattice shape,
model, precision, walls and repulsion so that every lattice of a shape runs the same
kernel (results then do not depend on what else was tuned or batched).
"""
from __future__ import annotations

import torch

from . import lbm

# tz = 0 selects the persistent grid (equal shares of all tile-planes per resident block)
CANDIDATES_3D = [(32, 8, 0), (32, 4, 0), (64, 4, 0), (16, 8, 0), (128, 2, 0),
                 (32, 8, 16), (32, 8, 22), (32, 8, 32), (32, 4, 16), (64, 4, 16),
                 (32, 16, 0), (64, 8, 0)]  # the last two: the ring kernel where it applies
CANDIDATES_2D = [(32, 8, 0), (32, 4, 0), (64, 4, 0), (128, 2, 0), (32, 8, 1), (32, 4, 1), (64, 4, 1), (128, 2, 1)]

_cache: dict = {}


def shape_key(lat: "lbm.Lattice"):
    p = lat.params
    return (p.lattice, p.model, p.precision, p.nx, p.ny, p.nz, getattr(lat, "_has_walls", False),
            p.model == lbm.CG and p.rep_pi != 0.0)


def candidates_for(p: "lbm.Params"):
    if p.streaming == lbm.STREAM_AA or p.model == lbm.SC_MR:
        return [(32, 8, 0)]  # the field-pass kernels choose their own launch shape
    cands = CANDIDATES_3D if p.lattice == lbm.D3Q19 else CANDIDATES_2D
    out = []
    for tx, ty, tz in cands:
        tz = min(tz, p.nz) if p.lattice == lbm.D3Q19 else tz
        if (tx, ty, tz) not in out:
            out.append((tx, ty, tz))
    return out


def time_steps(lat: "lbm.Lattice", steps: int) -> float:
    s = lat.stream
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    lat.step(steps)
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / steps


def autotune(lat: "lbm.Lattice", candidates=None, steps: int = 10, trials: int = 2, use_cache: bool = True):
    """Pick the fastest tiling for `lat` (state restored afterwards): each candidate is
    timed `trials` times over `steps` steps and keeps its best time, so that run-to-run
    noise of a few per cent does not flip close picks.  Returns
    (best tiling, {tiling: ms per step})."""
    key = shape_key(lat)
    if use_cache and key in _cache:
        lat.set_tiling(*_cache[key][0])
        return _cache[key]
    state = lat.save_state()
    solid = getattr(lat, "_solid", None)
    timings = {}
    for t in (candidates or candidates_for(lat.params)):
        try:
            lat.set_tiling(*t)
        except lbm.LbmError:
            continue
        lat.load_state(state, solid)
        lat.step(1)  # warm (first launch of a variant sets its shared-memory attribute)
        timings[t] = min(time_steps(lat, steps) for _ in range(trials))
    best = min(timings, key=timings.get)
    lat.set_tiling(*best)
    lat.load_state(state, solid)
    _cache[key] = (best, timings)
    return best, timings
