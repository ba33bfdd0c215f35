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
                 (32, 16, 0), (64, 8, 0),   # the ring kernel where it applies
                 (32, 8, 4), (32, 4, 4), (64, 4, 4)]  # short chunks: more units on small lattices
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


_batch_cache: dict = {}
BATCH_CHUNKS = (4, 8, 16)


def batch_chunk(p: "lbm.Params", copies: int = 8, steps: int = 20) -> int:
    """z planes per work unit for a lattice of these parameters in the batched launch
    (lbm_batch_*): times `copies` lattices of the shape, batched, for each chunk length in
    BATCH_CHUNKS and keeps the fastest (cached per shape, model and precision).  Shorter
    chunks give a small lattice more units; each unit also stages two halo planes.  The
    chunk length does not change results: every node is computed the same way."""
    import numpy as np
    key = (p.lattice, p.model, p.precision, p.nx, p.ny, p.nz)
    if p.lattice != lbm.D3Q19:
        return 1
    if key in _batch_cache:
        return _batch_cache[key]
    stream = torch.cuda.Stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(0)
    best, best_ms = BATCH_CHUNKS[-1], float("inf")
    for tz in BATCH_CHUNKS:
        if tz > p.nz:
            continue
        lats = []
        for _ in range(copies):
            lat = lbm.Lattice(p, stream=stream)
            rr = torch.as_tensor(1.0 + 0.01 * rng.standard_normal(p.n), device=dev)
            rb = None if p.model == lbm.SC_MP else torch.as_tensor(0.1 + 0.001 * rng.standard_normal(p.n), device=dev)
            with torch.cuda.stream(stream):
                lat.init(rr, rb)
            lat.set_tiling(32, 8, tz)
            lats.append(lat)
        b = lbm.Batch(p.precision, copies, 1 << 16, stream=stream)
        b.set(lats, [10 ** 6] * copies)
        b.step(steps)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b.step(steps)
        e.record(stream)
        e.synchronize()
        ms = a.elapsed_time(e)
        b.close()
        for lat in lats:
            lat.close()
        if ms < best_ms:
            best, best_ms = tz, ms
    _batch_cache[key] = best
    return best
