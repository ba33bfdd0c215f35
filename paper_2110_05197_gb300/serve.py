"""Serving loop for parameter sweeps: continuous batching of many simulations on one GPU.

A request is one simulation (grid, model, parameters, step count) arriving at some time.
Two servers answer the same request trace:

* ``PlainServer`` runs the requests one at a time in arrival order, FP32 storage, each
  lattice stepped with its own tuned kernel (the plain single-simulation path);
* ``BatchServer`` admits requests as they arrive while the device memory budget and the
  batch table have room, keeps their lattices resident, and advances all of them together:
  lattices up to ``batch_max_nodes`` nodes share one persistent batched launch per step
  (lbm_batch_*, replayed as a CUDA graph per tick of ``tick`` steps; each job's z-chunk
  length picked by the batch autotuner, tune.batch_chunk), larger ones are stepped with
  their own tuned kernel on ``big_streams`` further streams, one job per stream, in ticks
  of ``big_tick`` steps, so that several large lattices and the batch overlap on the
  device.  Every stream runs independently: an event marks its work in flight, and the
  host launches the next tick or job as soon as one completes.  A finished request's
  moments are read and its memory is released as soon as its work completes; new requests
  join at the next tick of their stream.

Results are the FP64 totals (lbm_moments) and the component densities; the latency of a
request is completion minus arrival on a common wall clock.  The physics of a job does
not depend on what else runs: the batched kernel computes every node with the same code
whatever the mix.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import inputs, lbm, tune

GRIDS = [(256, 256, 1), (32, 32, 32), (48, 48, 48), (64, 64, 64), (96, 96, 96)]


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the trace start
    grid: tuple             # (nx, ny, nz); nz == 1 is D2Q9
    model: int              # lbm.CG or lbm.SC_MP
    kw: dict                # lbm.Params fields besides lattice/model/precision/grid
    steps: int
    seed: int

    @property
    def nodes(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]

    def params(self, precision: int) -> "lbm.Params":
        nx, ny, nz = self.grid
        lat = lbm.D2Q9 if nz == 1 else lbm.D3Q19
        return lbm.Params(lattice=lat, model=self.model, precision=precision, nx=nx, ny=ny, nz=nz, **self.kw)


def sweep(n: int, seed: int = 5, steps=(5000, 20000), rate_hz: float = 1.0, grids=GRIDS) -> list:
    """Seeded request trace of a stability-map sweep: grid uniform over `grids`, CG or SC
    multiphase 50/50, density ratio log-uniform in [1, 1000], viscosity ratio log-uniform
    in [0.1, 10] (tau_B = 1, tau_R from nu_R), A log-uniform in [1e-4, 1e-1]; SC takes
    G uniform in the paper's stable window |G| in [4.2, 6.5] (its density ratio follows
    from G).  Step counts uniform in `steps`; Poisson arrivals at `rate_hz`."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate_hz)
        grid = grids[rng.integers(len(grids))]
        model = lbm.CG if rng.random() < 0.5 else lbm.SC_MP
        ratio = 10 ** rng.uniform(0, 3)
        nu_ratio = 10 ** rng.uniform(-1, 1)
        nu_b = 1 / 6
        tau_r = 3 * nu_ratio * nu_b + 0.5
        if model == lbm.CG:
            kw = dict(rho_r0=1.0, rho_b0=1.0 / ratio, tau_r=tau_r, tau_b=1.0, A=10 ** rng.uniform(-4, -1))
        else:
            kw = dict(G=-rng.uniform(4.2, 6.5), rho0_psi=1.0, tau_r=1.0)
        out.append(Request(rid, t, grid, model, kw, int(rng.integers(steps[0], steps[1] + 1)), seed * 100003 + rid))
    return out


def initial_fields(req: Request):
    """Centred droplet of radius L/4 with +-1% seeded noise (SC: liquid 2.0 / gas 0.15)."""
    nx, ny, nz = req.grid
    r = min(nx, ny) / 4 if nz == 1 else min(nx, ny, nz) / 4
    ins = inputs.sphere(nx, ny, nz, r)
    if req.model == lbm.CG:
        return inputs.two_fluid(ins, req.kw["rho_r0"], req.kw["rho_b0"], 0.01, req.seed)
    rho = np.where(ins, 2.0, 0.15) * (1 + 0.01 * inputs.uniform_pm1(req.seed, ins.size))
    return rho, None


@dataclass
class Result:
    rid: int
    arrival: float
    start: float
    done: float
    status: int
    totals: dict
    rho_r: np.ndarray = field(repr=False, default=None)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def _new_lattice(req: Request, precision: int, stream, tuned: bool):
    import torch
    lat = lbm.Lattice(req.params(precision), stream=stream)
    rr, rb = initial_fields(req)
    dev = lat.device
    t = lambda a: None if a is None else torch.as_tensor(a, dtype=torch.float64).to(dev, non_blocking=False)
    with torch.cuda.stream(stream):
        lat.init(t(rr), t(rb))
    if tuned:
        tune.autotune(lat)
    return lat


def _finish(lat, req, start, clock, keep_fields):
    rr = np.empty(req.nodes) if keep_fields else None
    tot = np.zeros(lbm.NTOTALS)
    rc = lat.moments_into(rr, None, None, None, tot)   # synchronises the stream
    return Result(req.rid, req.arrival, start, clock(), rc, dict(zip(lbm.TOTAL_NAMES, tot.tolist())), rr)


class PlainServer:
    """One request at a time, FP32 storage, the lattice's own tuned kernel."""

    def __init__(self, precision: int = lbm.FP32, keep_fields: bool = False):
        self.precision = precision
        self.keep_fields = keep_fields
        self.launches = 0

    def run(self, requests, t0=None):
        import torch
        stream = torch.cuda.Stream()
        t0 = time.perf_counter() if t0 is None else t0
        clock = lambda: time.perf_counter() - t0
        out = []
        for req in sorted(requests, key=lambda r: r.arrival):
            while clock() < req.arrival:
                time.sleep(min(1e-3, max(0.0, req.arrival - clock())))
            start = clock()
            lat = _new_lattice(req, self.precision, stream, tuned=True)
            l0 = lat.launch_count()
            lat.step(req.steps)
            self.launches += lat.launch_count() - l0
            out.append(_finish(lat, req, start, clock, self.keep_fields))
            lat.close()
        return out


class BatchServer:
    """Continuous batching with HBM-budget admission (see the module docstring)."""

    def __init__(self, precision: int = lbm.FP16, budget_bytes: int = 8 << 30, tick: int = 100,
                 max_jobs: int = 256, max_units: int = 1 << 16, batch_max_nodes: int = 120_000,
                 graph: bool = True, keep_fields: bool = False, big_streams: int = 4, big_tick: int = 500):
        self.precision = precision
        self.budget = budget_bytes
        self.tick = tick
        self.max_jobs = max_jobs
        self.max_units = max_units
        self.batch_max_nodes = batch_max_nodes
        self.graph = graph
        self.keep_fields = keep_fields
        self.big_streams = big_streams
        self.big_tick = big_tick
        self.launches = 0
        self.peak_bytes = 0
        self.peak_jobs = 0

    def run(self, requests, t0=None):
        import torch
        small_stream = torch.cuda.Stream()
        slots = [dict(stream=torch.cuda.Stream(), ev=None, job=None) for _ in range(self.big_streams)]
        batch = lbm.Batch(self.precision, self.max_jobs, self.max_units, stream=small_stream)
        t0 = time.perf_counter() if t0 is None else t0
        clock = lambda: time.perf_counter() - t0
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        smalls, bigs_waiting = [], deque()  # active jobs (dicts: req, lat, left, start, bytes, small, units)
        n_big_active = 0
        out = []
        used = 0
        units_used = 0
        dirty = False
        small_ev, small_running = None, []

        def finish(a):
            nonlocal used, units_used
            out.append(_finish(a["lat"], a["req"], a["start"], clock, self.keep_fields))
            a["lat"].close()
            used -= a["bytes"]
            units_used -= a["units"]

        while pending or smalls or bigs_waiting or n_big_active:
            now = clock()
            # admission: arrived requests, FIFO, while memory and table room remain
            while pending and pending[0].arrival <= now:
                req = pending[0]
                p = req.params(self.precision)
                need = lbm.workspace_bytes(p)
                small = req.nodes <= self.batch_max_nodes
                if used + need > self.budget or (small and len(smalls) >= self.max_jobs):
                    break
                if small:
                    # the batch stream: its job's z-chunk from the batch autotuner
                    lat = _new_lattice(req, self.precision, small_stream, tuned=False)
                    lat.set_tiling(32, 8, tune.batch_chunk(req.params(self.precision)))
                    nu = lbm.Batch.units(lat)
                    if units_used + nu > self.max_units:
                        lat.close()
                        break
                    pending.popleft()
                    smalls.append(dict(req=req, lat=lat, left=req.steps, start=now, bytes=need, small=True, units=nu))
                    units_used += nu
                    dirty = True
                else:
                    pending.popleft()
                    bigs_waiting.append(dict(req=req, lat=None, left=req.steps, start=now, bytes=need, small=False,
                                             units=0))
                used += need
            self.peak_bytes = max(self.peak_bytes, used)
            self.peak_jobs = max(self.peak_jobs, len(smalls) + n_big_active + len(bigs_waiting))
            progressed = False
            # small lattices: one batched launch per step, ticks of `tick` steps as a graph;
            # the job list changes only between ticks
            if small_ev is None or small_ev.query():
                if small_ev is not None:
                    for a in small_running:
                        a["left"] -= min(self.tick, a["left"])
                        if a["left"] == 0:
                            smalls.remove(a)
                            finish(a)
                            dirty = True
                    small_ev, small_running = None, []
                    progressed = True
                if smalls:
                    if dirty:
                        batch.set([a["lat"] for a in smalls], [a["left"] for a in smalls])
                        dirty = False
                    batch.step(self.tick, graph=self.graph)
                    small_ev = torch.cuda.Event()
                    small_ev.record(small_stream)
                    small_running = list(smalls)
            # large lattices: one job per stream slot, ticks of `big_tick` steps
            for sl in slots:
                if sl["ev"] is not None and not sl["ev"].query():
                    continue
                a = sl["job"]
                if a is not None and a["left"] == 0:
                    finish(a)
                    sl["job"], a = None, None
                    n_big_active -= 1
                    progressed = True
                if a is None and bigs_waiting:
                    a = bigs_waiting.popleft()
                    a["lat"] = _new_lattice(a["req"], self.precision, sl["stream"], tuned=True)
                    sl["job"] = a
                    n_big_active += 1
                if a is not None:
                    k = min(self.big_tick, a["left"])
                    l0 = a["lat"].launch_count()
                    a["lat"].step(k)
                    self.launches += a["lat"].launch_count() - l0
                    a["left"] -= k
                    sl["ev"] = torch.cuda.Event()
                    sl["ev"].record(sl["stream"])
                    progressed = True
                else:
                    sl["ev"] = None
            if not progressed:
                if small_ev is None and not n_big_active and pending:
                    time.sleep(min(1e-3, max(0.0, pending[0].arrival - clock())))
                else:
                    time.sleep(2e-5)
        self.launches += batch.launch_count()
        batch.close()
        return out


def summary(results) -> dict:
    lat = np.array([r.latency for r in results])
    makespan = max(r.done for r in results) - min(r.arrival for r in results)
    return {"requests": len(results), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "sims_per_hour": len(results) / makespan * 3600.0, "makespan_s": makespan,
            "unstable": int(sum(r.status != lbm.OK for r in results))}
