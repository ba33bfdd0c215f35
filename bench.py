#!/usr/bin/env python3
"""Benchmark of the two-component LBM step on GB300 (D3Q19 CG and SC oscillating droplet).

Workload (one "step"): one colour-gradient timestep of a 128^3 D3Q19 lattice (ellipsoidal
droplet, semi-axes 24/20/20, density ratio 10, A = 5e-3, tau = 1, +-1% seeded noise) and one
Shan-Chen multiphase timestep of a 128^3 D3Q19 lattice (same ellipsoid, G = -5, rho_0 = 1),
both FP32.  value = lattice updates of both lattices per second (MLUPS); both lattices'
populations (318 MB + 159 MB) exceed the 126 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own pair of lattices (independent replicas, weak
scaling); rank 0 prints one JSON line with the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2110_05197_gb300 import inputs  # noqa: E402

METRIC = "CG/SC D3Q19 MLUPS & % HBM roofline; sweep sims/hr + p99 latency vs plain"
N3 = 128
SEMI = (24.0, 20.0, 20.0)
SC_LIQ, SC_GAS = 1.8884, 0.1194          # SC coexistence at G = -5 (mechanical stability)
BYTES_PER_LU = {"cg": 2 * 2 * 19 * 4, "sc": 2 * 1 * 19 * 4}   # FP32 read + write of all populations
FALLBACK_HBM_GBS = 6800.0


def workload_fields(n=N3, nz=None):
    nz = nz or n
    ins = inputs.ellipsoid(n, n, nz, SEMI, centre=((n - 1) / 2, (n - 1) / 2, (nz - 1) / 2))
    rr, rb = inputs.two_fluid(ins, 1.0, 0.1, 0.01, 2)
    rho_sc = np.where(ins, SC_LIQ, SC_GAS) * (1 + 0.01 * inputs.uniform_pm1(2, ins.size))
    return rr, rb, rho_sc


def cg_kw(n=N3, nz=None):
    return dict(lattice=1, model=0, nx=n, ny=n, nz=nz or n, rho_r0=1.0, rho_b0=0.1, alpha_b=0.2,
                tau_r=1.0, tau_b=1.0, A=5e-3, beta=0.7)


def sc_kw(n=N3, nz=None):
    return dict(lattice=1, model=1, nx=n, ny=n, nz=nz or n, G=-5.0, rho0_psi=1.0, tau_r=1.0)


# Sources that define the FP32 step kernels and their launch (the profiled kernels).
STEP_KERNEL_SOURCES = ("lbm_lattice.cuh", "lbm_rep.cuh", "lbm_step.cuh", "lbm_step_tma.cuh", "lbm_step_tmac.cuh",
                       "lbm_step_ring.cuh", "lbm_launch.cuh", "lbm_internal.cuh", "lbm_step_f32.cu")


def csrc_sha256_16():
    """Hash of the step kernels' CUDA sources (the kernels whose counters a profile records)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2110_05197_gb300", "csrc")
    for name in STEP_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary under profiles/,
    or None when no summary exists or the kernel sources changed since it was taken."""
    import glob
    sha = csrc_sha256_16()
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(path) as f:
            for line in f:
                if not line.startswith("roofline-traffic:"):
                    continue
                kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
                if kv.get("kernel") == kernel and kv.get("csrc_sha256_16") == sha:
                    return int(kv["bytes_per_launch"])
    return None


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
            if k in d:
                return float(d[k]), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling (every 200 ms, each sample time-stamped by
    nvidia-smi itself).  summary() keeps the samples inside the marked timed region; when
    that region is shorter than a few sampling periods it widens the window to the load
    phase marked just before it (the same steps, untimed) and says so."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.marks = {}

    def mark(self, name: str):
        self.marks[name] = time.time()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def _samples(self):
        import datetime
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        out = []
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm, mx = float(f[2]), float(f[3])
            except ValueError:
                continue
            out.append((ts, sm, mx, {nm for nm, v in zip(names, f[6:10]) if v.lower() == "active"}))
        return out

    def summary(self, start="timed_start", end="timed_end", wide_start="load_start"):
        samples = self._samples()
        t0, t1 = self.marks.get(start), self.marks.get(end)
        window = "timed region"
        sel = [s for s in samples if t0 is not None and t1 is not None and t0 <= s[0] <= t1]
        if len(sel) < 3 and wide_start in self.marks:
            window = "timed region + the untimed load phase of the same steps just before it"
            sel = [s for s in samples if self.marks[wide_start] <= s[0] <= (t1 or s[0])]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = set().union(*(s[3] for s in sel))
        return {"sm_mhz": statistics.median(s[1] for s in sel), "sm_max_mhz": max(s[2] for s in sel),
                "reasons": sorted(reasons), "samples": len(sel), "window": window}


def slowest_rank(value: float, device=None) -> float:
    """Max of a per-rank time over all ranks (the job's time is the slowest replica's);
    the identity without a process group.  device: where the collective's tensor lives
    (a CUDA device under NCCL, None = CPU under gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes_per_rank: int, lattices: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas (weak scaling): every rank advances its
    own `lattices` lattices of `nodes_per_rank` nodes by `steps` steps; `seconds` is the
    slowest rank's time."""
    return lattices * nodes_per_rank * steps * world / seconds / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample_mlups(steps: int, nz: int = 16, threads: int | None = None, budget_s: float | None = None):
    """FP64 CPU oracle on a 128 x 128 x nz slab of the same droplet workload (CG + SC).
    With budget_s, steps is the minimum and the loop runs on until budget_s seconds
    (bounded CPU work); returns (MLUPS, threads, seconds, nodes per lattice, steps)."""
    import oracle
    oracle.build()
    threads = threads or os.cpu_count() or 1
    oracle.set_threads(threads)
    rr, rb, rho = workload_fields(N3, nz)
    cg = oracle.OracleSim(oracle.Params(**cg_kw(N3, nz))).init(rr, rb)
    sc = oracle.OracleSim(oracle.Params(**sc_kw(N3, nz))).init(rho)
    n = N3 * N3 * nz
    t0 = time.perf_counter()
    done = 0
    while done < steps or (budget_s is not None and time.perf_counter() - t0 < budget_s):
        cg.step(1)
        sc.step(1)
        done += 1
    dt = time.perf_counter() - t0
    return 2 * n * done / dt / 1e6, oracle.get_threads(), dt, n, done


def serving_sweep(n_req: int, seed: int = 5):
    """Continuous-batching sweep at the stated step range: stability-map requests over 2D
    256^2 and 32^3..96^3 grids, CG or SC, 5000-20000 steps each (`n_req` of the 512
    requests of the full sweep, seeded; nothing is extrapolated).  First a closed batch
    (every request at t = 0) through the plain FP32 one-at-a-time server measures its
    service rate mu; then one Poisson trace at 1.2 mu is replayed through both servers."""
    import torch
    from paper_2110_05197_gb300 import lbm, serve
    # tune every grid shape and model once for both servers (tiling and batch chunk caches)
    warm = [serve.Request(i, 0.0, g, m, kw, 5, 1) for i, (g, m, kw) in enumerate(
        (g, m, dict(rho_r0=1.0, rho_b0=0.1, tau_r=1.0, tau_b=1.0, A=1e-2) if m == lbm.CG else
         dict(G=-5.0, rho0_psi=1.0, tau_r=1.0)) for g in serve.GRIDS for m in (lbm.CG, lbm.SC_MP))]
    serve.PlainServer(lbm.FP32).run(warm)
    serve.BatchServer(lbm.FP16, tick=100).run(warm)
    torch.cuda.synchronize()
    steps = (5000, 20000)
    closed = serve.sweep(n_req, seed=seed, steps=steps, rate_hz=1e6)
    out = {"requests": n_req, "of_requests": 512, "steps": f"U[{steps[0]}, {steps[1]}] per request (the stated range)",
           "grids": [list(g) for g in serve.GRIDS], "precision": {"plain": "fp32", "batch": "fp16 storage"}}
    res_plain_closed = serve.PlainServer(lbm.FP32).run(closed)
    res_batch_closed = serve.BatchServer(lbm.FP16, tick=100).run(closed)
    pc, bc = serve.summary(res_plain_closed), serve.summary(res_batch_closed)
    out["closed_batch"] = {"plain_fp32": pc, "batch_fp16": bc, "sims_per_hour_ratio": bc["sims_per_hour"] / pc["sims_per_hour"]}
    mu = n_req / pc["makespan_s"]
    trace = serve.sweep(n_req, seed=seed, steps=steps, rate_hz=1.2 * mu)
    plain_srv, batch_srv = serve.PlainServer(lbm.FP32), serve.BatchServer(lbm.FP16, tick=100)
    pp = serve.summary(plain_srv.run(trace))
    bb = serve.summary(batch_srv.run(trace))
    out["poisson"] = {"rate_hz": 1.2 * mu, "plain_fp32": pp, "batch_fp16": bb,
                      "sims_per_hour_ratio": bb["sims_per_hour"] / pp["sims_per_hour"],
                      "batch_peak_resident_jobs": batch_srv.peak_jobs,
                      "batch_peak_workspace_bytes": batch_srv.peak_bytes,
                      "launches": {"plain": plain_srv.launches, "batch": batch_srv.launches}}
    return out


def kernel_label(model: str, precision: int, tiling) -> str:
    """The step kernel a tiling runs on the 128^3 benchmark lattices (nx / tx <= 8): the
    ring kernel for 32 x 16 and 64 x 8 tiles, and for 64 x 4 tiles where two of its blocks
    fit an SM (SC multiphase, or 16-bit storage); the cluster TMA kernel for the other
    32 x 8, 32 x 4 and 64 x 4 tiles; the generic kernel otherwise.  The label names the
    tile, whose traffic differs."""
    tx, ty = int(tiling[0]), int(tiling[1])
    elt = {1: "float", 2: "half", 3: "bf16"}[precision]
    m = "CG" if model == "cg" else "SC-MP"
    ring = (tx, ty) in ((32, 16), (64, 8)) or ((tx, ty) == (64, 4) and (model == "sc" or precision != 1))
    if ring and not (model == "cg" and precision == 1 and tx == 64):
        return f"step_kernel_ring<D3Q19,{elt},{m},{tx}x{ty}>"
    if (tx, ty) in ((32, 8), (32, 4), (64, 4)):
        return f"step_kernel_tmac<D3Q19,{elt},{m},{tx}x{ty}>"
    return f"step_kernel<D3Q19,{elt},{m}>"


def storage16_steps(rr, rb, rho, dev, stream, steps: int = 20):
    """Step times of the same two lattices with FP16 storage of the shifted populations
    (FP32 arithmetic), each on its autotuned tiling, with the fraction of the measured HBM
    bandwidth at their algorithmic bytes (152 B/LU CG, 76 B/LU SC; not part of `value`)."""
    import torch
    from paper_2110_05197_gb300 import lbm, tune
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    peak, _ = hbm_peak()
    out = {"bytes_per_lu": {"cg": 2 * 19 * 2 * 2, "sc": 19 * 2 * 2}}
    for name, kw, fields in (("cg", cg_kw(), (rr, rb)), ("sc", sc_kw(), (rho,))):
        lat = lbm.Lattice(lbm.Params(precision=lbm.FP16, **kw), stream=stream)
        lat.init(*(t(f) for f in fields))
        best, _ = tune.autotune(lat)
        lat.step(3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.step(steps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        gbs = out["bytes_per_lu"][name] * N3 ** 3 / (ms / 1e3) / 1e9
        out[name] = {"step_ms": ms, "mlups": N3 ** 3 / (ms / 1e3) / 1e6, "achieved_gbs": gbs,
                     "frac": gbs / peak, "tiling": list(best), "kernel": kernel_label(name, lbm.FP16, best),
                     "status": lbm.status_string(lat.totals()[1])}
        lat.close()
    return out


def emulsion_steps(dev, stream, steps: int = 10):
    """Step times of the dense emulsion with the CG repulsion force (256^3 periodic, 200
    droplets of radius 10 +- 2, Table emulsionParams: rho 1.36, A 0.0518, Pi 0.012, chi 2),
    FP32 and FP16 storage, autotuned; MLUPS and the fraction of the measured HBM bandwidth
    at the algorithmic bytes (304 / 152 B/LU; the repulsion pre-pass's colour and normal
    fields are implementation traffic).  Not part of `value`."""
    import torch
    from paper_2110_05197_gb300 import lbm, tune
    n = 256
    ins, _ = inputs.emulsion(n, n, n, count=200, r_mean=10.0, r_spread=2.0, gap=3.0, seed=4)
    rr, rb = inputs.two_fluid(ins, 1.36, 1.36, 0.01, 5)
    kw = dict(lattice=1, model=0, nx=n, ny=n, nz=n, rho_r0=1.36, rho_b0=1.36, A=0.0518, rep_pi=0.012, rep_chi=2.0,
              grad_eps=1e-4)
    peak, _ = hbm_peak()
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    out = {"workload": "CG dense emulsion with the repulsion force, 256^3, 200 droplets", "steps": steps}
    for name, prec, bpl in (("fp32", lbm.FP32, 304), ("fp16", lbm.FP16, 152)):
        lat = lbm.Lattice(lbm.Params(precision=prec, **kw), stream=stream)
        lat.init(t(rr), t(rb))
        best, _ = tune.autotune(lat, steps=3, trials=1)
        lat.step(2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.step(steps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        gbs = bpl * n ** 3 / (ms / 1e3) / 1e9
        out[name] = {"step_ms": ms, "mlups": n ** 3 / (ms / 1e3) / 1e6, "bytes_per_lu": bpl, "achieved_gbs": gbs,
                     "frac": gbs / peak, "tiling": list(best), "status": lbm.status_string(lat.totals()[1])}
        lat.close()
        torch.cuda.empty_cache()
    return out


def in_place_steps(rr, rb, rho, dev, stream, steps: int = 20):
    """Step times of the same two lattices with in-place (AA) streaming: one population
    buffer, a field pass plus the step kernel per step (not part of `value`)."""
    import torch
    from paper_2110_05197_gb300 import lbm
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    out = {"bytes_moved_per_lu": {"cg": 2 * 19 * 4 + 8 + 16 + 2 * (2 * 19 * 4 + 8) + 16,
                                  "sc": 19 * 4 + 4 + 8 + 2 * (19 * 4 + 4) + 8}}
    for name, kw, fields in (("cg", cg_kw(), (rr, rb)), ("sc", sc_kw(), (rho,))):
        lat = lbm.Lattice(lbm.Params(precision=lbm.FP32, streaming=lbm.STREAM_AA, **kw), stream=stream)
        lat.init(*(t(f) for f in fields))
        lat.step(3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.step(steps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        out[f"{name}_step_ms"] = ms
        out[f"{name}_mlups"] = N3 ** 3 / (ms / 1e3) / 1e6
        out[f"{name}_status"] = lbm.status_string(lat.totals()[1])
        lat.close()
    return out


def multirange_steps(dev, stream, steps: int = 20):
    """Step time of the multicomponent SC model with multirange potentials on a 128^3 box
    (a drop of species A; Table dropcolParams couplings with G_AB read as 1.215), FP32,
    two buffers: the field pass plus the belt-2 step kernel (not part of `value`)."""
    import torch
    from paper_2110_05197_gb300 import lbm
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    ins = inputs.sphere(N3, N3, N3, N3 / 4)
    kw = dict(lattice=1, model=lbm.SC_MR, nx=N3, ny=N3, nz=N3, Ga=(-9.0, -8.0), Gr=(8.1, 7.1), G=1.215,
              rho0_psi=0.83)
    lat = lbm.Lattice(lbm.Params(precision=lbm.FP32, **kw), stream=stream)
    lat.init(t(np.where(ins, 1.18, 0.18)), t(np.where(ins, 0.18, 1.18)))
    lat.step(3)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    lat.step(steps)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    out = {"step_ms": ms, "mlups": N3 ** 3 / (ms / 1e3) / 1e6, "bytes_per_lu": BYTES_PER_LU["cg"],
           "frac_of_hbm": BYTES_PER_LU["cg"] * N3 ** 3 / (ms / 1e3) / 1e9 / hbm_peak()[0],
           "status": lbm.status_string(lat.totals()[1])}
    lat.close()
    return out


def workload_config(ws: int) -> dict:
    """The benchmark workload, the same for both arms (the reference arm times a slab of it,
    stated in its cpu_baseline sample)."""
    return {"workload": "D3Q19 CG + SC multiphase oscillating droplet, 128^3 each, FP32",
            "lattice": "D3Q19", "nx": N3, "ny": N3, "nz": N3, "density_ratio": 10,
            "cg": {"A": 5e-3, "tau": 1.0, "beta": 0.7}, "sc": {"G": -5.0, "rho0": 1.0, "tau": 1.0},
            "l2": "inputs larger than L2 (477 MB of populations per step)",
            "parallelism": f"replicas x{ws}"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    nz = 32
    oracle_sample_mlups(max(1, args.warmup), nz)
    mlups, cores, dt, n, _ = oracle_sample_mlups(args.steps, nz)
    sample = f"128x128x{nz} slab of the 128^3 droplet workload, CG + SC FP64 oracle, {args.steps} steps"
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(1),
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2110_05197_gb300 import build, lbm
    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    rr, rb, rho = workload_fields()
    n = N3 ** 3
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    cg = lbm.Lattice(lbm.Params(precision=lbm.FP32, **cg_kw()))
    sc = lbm.Lattice(lbm.Params(precision=lbm.FP32, **sc_kw()))
    cg.init(t(rr), t(rb))
    sc.init(t(rho))
    from paper_2110_05197_gb300 import tune
    tiling = {}
    if args.tiling:
        tx, ty, tz = (int(v) for v in args.tiling.split(","))
        cg.set_tiling(tx, ty, tz)
        sc.set_tiling(tx, ty, tz)
        tiling = {"cg": [tx, ty, tz], "sc": [tx, ty, tz], "tuned": False}
    else:
        best_cg, tm_cg = tune.autotune(cg)
        best_sc, tm_sc = tune.autotune(sc)
        tiling = {"cg": list(best_cg), "sc": list(best_sc), "tuned": True,
                  "cg_ms": {"x".join(map(str, k)): round(v, 4) for k, v in tm_cg.items()},
                  "sc_ms": {"x".join(map(str, k)): round(v, 4) for k, v in tm_sc.items()}}
    if args.profile_only in ("mr", "aa_cg", "aa_sc"):
        # the field-pass kernels on the same 128^3 box: the multirange SC model (a drop of
        # species A, Table dropcolParams couplings with the cross coupling read as 1.215) or
        # the benchmark lattices with in-place streaming
        if args.profile_only == "mr":
            ins = inputs.sphere(N3, N3, N3, N3 / 4)
            kw = dict(lattice=1, model=3, nx=N3, ny=N3, nz=N3, Ga=(-9.0, -8.0), Gr=(8.1, 7.1), G=1.215,
                      rho0_psi=0.83)
            lat = lbm.Lattice(lbm.Params(precision=lbm.FP32, **kw))
            lat.init(t(np.where(ins, 1.18, 0.18)), t(np.where(ins, 0.18, 1.18)))
        elif args.profile_only == "aa_cg":
            lat = lbm.Lattice(lbm.Params(precision=lbm.FP32, streaming=lbm.STREAM_AA, **cg_kw()))
            lat.init(t(rr), t(rb))
        else:
            lat = lbm.Lattice(lbm.Params(precision=lbm.FP32, streaming=lbm.STREAM_AA, **sc_kw()))
            lat.init(t(rho))
        lat.step(args.warmup + args.steps)
        torch.cuda.synchronize()
        return 0
    if args.profile_only:
        lat = cg if args.profile_only == "cg" else sc
        lat.step(args.warmup + args.steps)
        torch.cuda.synchronize()
        return 0
    for _ in range(args.warmup):
        cg.step(1)
        sc.step(1)
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        # untimed load phase (>= 1.2 s of the same steps) so that the clock record has
        # samples under load even when K steps take only milliseconds
        clk.mark("load_start")
        t_load = time.perf_counter()
        while time.perf_counter() - t_load < 1.2:
            for _ in range(20):
                cg.step(1)
                sc.step(1)
            torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = cg.launch_count() + sc.launch_count()
        clk.mark("timed_start")
        start.record(stream)
        for k in range(K):
            ev[k][0].record(stream)
            cg.step(1)
            ev[k][1].record(stream)
            sc.step(1)
            ev[k][2].record(stream)
        end.record(stream)
        torch.cuda.synchronize()
        clk.mark("timed_end")
    launches = cg.launch_count() + sc.launch_count() - l0
    total_ms = slowest_rank(start.elapsed_time(end), dev)
    cg_ms = [a.elapsed_time(b) for a, b, _ in ev]
    sc_ms = [b.elapsed_time(c) for _, b, c in ev]
    cg_avg, sc_avg = float(np.mean(cg_ms)), float(np.mean(sc_ms))
    value = job_mlups(n, 2, K, ws, total_ms / 1e3)
    peak, peak_kind = hbm_peak()
    cg_kernel = kernel_label("cg", lbm.FP32, tiling["cg"])
    sc_kernel = kernel_label("sc", lbm.FP32, tiling["sc"])
    achieved = BYTES_PER_LU["cg"] * n / (cg_avg / 1e3) / 1e9
    tot_cg, rc_cg = cg.totals()
    tot_sc, rc_sc = sc.totals()
    in_place = in_place_steps(rr, rb, rho, dev, stream)
    storage16 = storage16_steps(rr, rb, rho, dev, stream)
    emulsion = emulsion_steps(dev, stream)
    multirange = multirange_steps(dev, stream)

    # end to end through the public API with pinned host buffers: init from host fields,
    # K CG + K SC steps, densities and totals back to the host
    pin = lambda a: torch.as_tensor(a, dtype=torch.float64).pin_memory()
    h_rr, h_rb, h_rho = pin(rr), pin(rb), pin(rho)
    o_rr, o_rb, o_sc = (torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(3))
    totals = np.zeros(lbm.NTOTALS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cg.init(h_rr, h_rb)
    sc.init(h_rho)
    cg.step(K)
    sc.step(K)
    cg.moments_into(o_rr, o_rb, None, None, totals)
    sc.moments_into(o_sc, None, None, None, totals)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = 3 * n * 8
    d2h = 3 * n * 8 + 2 * lbm.NTOTALS * 8
    e2e_mlups = job_mlups(n, 2, K, ws, slowest_rank(e2e_s, dev))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": workload_config(ws),
            "cg_mlups": n / (cg_avg / 1e3) / 1e6, "sc_mlups": n / (sc_avg / 1e3) / 1e6,
            "cg_step_ms": cg_avg, "sc_step_ms": sc_avg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": profiled_traffic(cg_kernel),
                         "kernel": cg_kernel,
                         "bytes_per_lu": BYTES_PER_LU["cg"], "peak_kind": peak_kind,
                         "sc": {"achieved": BYTES_PER_LU["sc"] * n / (sc_avg / 1e3) / 1e9,
                                "frac": BYTES_PER_LU["sc"] * n / (sc_avg / 1e3) / 1e9 / peak,
                                "kernel": sc_kernel, "bytes_per_lu": BYTES_PER_LU["sc"],
                                "traffic": profiled_traffic(sc_kernel)}},
            "clocks": clk.summary(),
            "e2e": {"value": e2e_mlups, "unit": "MLUPS", "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
                    "request": f"init from pinned host fields + {K} CG and {K} SC steps + densities/totals to host"},
            "gpu_launches": launches,
            "tiling": tiling,
            "in_place": in_place,
            "fp16_storage": storage16,
            "emulsion": emulsion,
            "multirange": multirange,
            "status": {"cg": lbm.status_string(rc_cg), "sc": lbm.status_string(rc_sc),
                       "cg_mass_r": tot_cg["mass_r"], "sc_mass": tot_sc["mass_r"]},
        }
        if not args.no_serving and ws == 1:
            line["serving"] = serving_sweep(args.serving_requests)
        if not args.no_cpu_baseline:
            mlups_cpu, cores, dt, ns, done = oracle_sample_mlups(1, N3, budget_s=10.0)
            line["cpu_baseline"] = {"value": mlups_cpu, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                    "sample": f"FP64 oracle, {done} CG + {done} SC steps of the full 128^3 "
                                              f"workload ({dt:.1f} s)"}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tiling", default=None, help="tx,ty,tz for both lattices (default: autotuned)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving sweep")
    ap.add_argument("--serving-requests", type=int, default=32,
                    help="requests of the 512-request serving sweep to run at the full 5k-20k step range")
    ap.add_argument("--profile-only", default=None, choices=["cg", "sc", "mr", "aa_cg", "aa_sc"],
                    help="profiling runs: warm up and step only this lattice, print nothing")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
