"""Python binding of liblbm.so (include/lbm.h): argument marshalling only.

Every step of the lattice update runs in the CUDA library.  PyTorch supplies the device
workspace and the stream; nothing here computes on the lattice.  Importing this module
does not load the library; the first :class:`Lattice` (or :func:`lib`) does, and raises
if the library is missing or cannot be loaded -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, fields

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

D2Q9, D3Q19 = 0, 1
CG, SC_MP, SC_2C, SC_MR = 0, 1, 2, 3
FP64, FP32, FP16, BF16 = 0, 1, 2, 3
STREAM_AB, STREAM_AA = 0, 1
NTOTALS = 10
TOTAL_NAMES = ("mass_r", "mass_b", "mom_x", "mom_y", "mom_z", "e_kin", "max_u", "nonfinite",
               "min_rho_r", "min_rho_b")

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ESTATE, ETIMEOUT = range(7)


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class _CParams(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("model", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("rho_r0", ctypes.c_double), ("rho_b0", ctypes.c_double), ("alpha_b", ctypes.c_double),
        ("tau_r", ctypes.c_double), ("tau_b", ctypes.c_double),
        ("A", ctypes.c_double), ("beta", ctypes.c_double),
        ("enhanced_eq", ctypes.c_int32), ("color_norm", ctypes.c_int32),
        ("rep_pi", ctypes.c_double), ("rep_chi", ctypes.c_double),
        ("rep_psi_kind", ctypes.c_int32),
        ("grad_eps", ctypes.c_double),
        ("G", ctypes.c_double), ("rho0_psi", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("diag_every", ctypes.c_int32),
        ("umax_unstable", ctypes.c_double),
        ("streaming", ctypes.c_int32),
        ("Ga", ctypes.c_double * 2), ("Gr", ctypes.c_double * 2),
    ]


# exported symbol -> (restype, argtypes)
_VP = ctypes.c_void_p
SIGNATURES = {
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(_CParams), _VP, ctypes.POINTER(ctypes.c_size_t), _VP,
                                  ctypes.POINTER(_VP)]),
    "lbm_init_fields": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "lbm_step_cg": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "lbm_step_sc": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "lbm_moments": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "lbm_destroy": (ctypes.c_int, [_VP]),
    "lbm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_set_tiling": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "lbm_launch_count": (ctypes.c_uint64, [_VP]),
    "lbm_state_bytes": (ctypes.c_size_t, [_VP]),
    "lbm_save_state": (ctypes.c_int, [_VP, _VP]),
    "lbm_load_state": (ctypes.c_int, [_VP, _VP, _VP]),
    "lbm_totals_noalloc": (ctypes.c_int, [ctypes.POINTER(_CParams), _VP, _VP, _VP, _VP]),
    "lbm_state_planes_bytes": (ctypes.c_size_t, [_VP, ctypes.c_int32]),
    "lbm_get_state_planes": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP]),
    "lbm_set_state_planes": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP,
                                        ctypes.POINTER(ctypes.c_size_t), _VP, ctypes.POINTER(_VP)]),
    "lbm_batch_units": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32)]),
    "lbm_batch_set": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "lbm_batch_step": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32]),
    "lbm_batch_launch_count": (ctypes.c_uint64, [_VP]),
    "lbm_batch_destroy": (ctypes.c_int, [_VP]),
}
NOALLOC_MAX_NODES = 1 << 20


def _noalloc_args(params: "Params", pops, solid, out, stream):
    """Check what lbm_totals_noalloc cannot check itself (it gets raw pointers): dtypes,
    contiguity, sizes and that every device tensor is on the current device."""
    import torch

    def bad(why):
        raise LbmError(EINVAL, f"lbm_totals_noalloc: {why}")

    if not isinstance(pops, torch.Tensor) or not pops.is_cuda:
        bad("pops must be a CUDA tensor")
    dev = torch.cuda.current_device()
    if pops.device.index != dev:
        bad(f"pops is on cuda:{pops.device.index}, the current device is cuda:{dev}")
    if pops.dtype != torch.float64 or not pops.is_contiguous():
        bad("pops must be a contiguous float64 tensor")
    if pops.numel() < params.ncomp * params.q * params.n:
        bad(f"pops holds {pops.numel()} values, K*Q*N = {params.ncomp * params.q * params.n}")
    if solid is not None:
        if not isinstance(solid, torch.Tensor) or not solid.is_cuda or solid.device.index != dev:
            bad("solid must be a CUDA tensor on the current device")
        if solid.dtype != torch.uint8 or not solid.is_contiguous() or solid.numel() < params.n:
            bad("solid must be a contiguous uint8 tensor of N values")
    if isinstance(out, torch.Tensor):
        if not out.is_cuda or out.device.index != dev or out.dtype != torch.float64 or \
                not out.is_contiguous() or out.numel() < NTOTALS:
            bad("a device out must be a contiguous float64 CUDA tensor of NTOTALS values on the current device")
    elif not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous and
              out.size >= NTOTALS):
        bad("a host out must be a contiguous float64 array of NTOTALS values")
    if stream is not None and stream.device.index != dev:
        bad("the stream belongs to another device")


def totals_noalloc(params: "Params", pops, solid=None, out=None, stream=None):
    """lbm_totals_noalloc: totals of caller-owned canonical FP64 populations on the device,
    using the library's static scratch (no allocation).  Returns (totals, status).
    Raises LbmError(EINVAL) for a wrong dtype, size, layout or device before the call."""
    cp = params.to_c()
    if out is None:
        out = np.zeros(NTOTALS)
    _noalloc_args(params, pops, solid, out, stream)
    s = stream.cuda_stream if stream is not None else None
    rc = lib().lbm_totals_noalloc(ctypes.byref(cp), _ptr(pops), _ptr(solid), _ptr(out), s)
    if rc not in (OK, EUNSTABLE):
        raise LbmError(rc, "lbm_totals_noalloc")
    return out, rc

def workspace_bytes(params: "Params") -> int:
    """Device workspace lbm_create needs for these parameters (size query, no allocation)."""
    cp = params.to_c()
    need = ctypes.c_size_t(0)
    _check(lib().lbm_create(ctypes.byref(cp), None, ctypes.byref(need), None, None), "lbm_create(size)")
    return int(need.value)


_lib = None


def lib(path: str = LIB_PATH):
    """Load liblbm.so (raises OSError if it is missing: build it with build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"liblbm.so not found at {path}; run paper_2110_05197_gb300.build")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(s: int) -> str:
    try:
        return lib().lbm_status_string(int(s)).decode()
    except OSError:
        return f"status {s}"


def _check(rc: int, where: str):
    if rc != OK:
        raise LbmError(rc, where)


@dataclass
class Params:
    """Mirror of lbm_params (include/lbm.h)."""
    lattice: int = D3Q19
    model: int = CG
    precision: int = FP32
    nx: int = 16
    ny: int = 16
    nz: int = 16
    rho_r0: float = 1.0
    rho_b0: float = 1.0
    alpha_b: float = 0.2
    tau_r: float = 1.0
    tau_b: float = 1.0
    A: float = 1e-2
    beta: float = 0.7
    enhanced_eq: int = 1
    color_norm: int = 0
    rep_pi: float = 0.0
    rep_chi: float = 2.0
    rep_psi_kind: int = 0
    grad_eps: float = 0.0
    G: float = 0.0
    rho0_psi: float = 1.0
    body_force: tuple = (0.0, 0.0, 0.0)
    diag_every: int = 0
    umax_unstable: float = 0.5
    streaming: int = 0          # STREAM_AB (two buffers) or STREAM_AA (in place)
    Ga: tuple = (0.0, 0.0)      # SC_MR: attractive self-couplings per species
    Gr: tuple = (0.0, 0.0)      # SC_MR: repulsive self-couplings per species

    def to_c(self) -> _CParams:
        p = _CParams()
        for f in fields(self):
            v = getattr(self, f.name)
            if f.name in ("body_force", "Ga", "Gr"):
                setattr(p, f.name, (ctypes.c_double * len(v))(*[float(x) for x in v]))
            else:
                setattr(p, f.name, v)
        return p

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def q(self) -> int:
        return 19 if self.lattice == D3Q19 else 9

    @property
    def ncomp(self) -> int:
        return 1 if self.model == SC_MP else 2


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Lattice:
    """One lattice on the current CUDA device, with its workspace held as a torch tensor."""

    def __init__(self, params: Params, stream=None, device=None):
        import torch
        self.params = params
        self._cp = params.to_c()
        L = lib()
        need = ctypes.c_size_t(0)
        _check(L.lbm_create(ctypes.byref(self._cp), None, ctypes.byref(need), None, None), "lbm_create(size)")
        self.ws_bytes = need.value
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=dev)
        base = self.ws.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        h = ctypes.c_void_p()
        got = ctypes.c_size_t(self.ws_bytes)
        _check(L.lbm_create(ctypes.byref(self._cp), ctypes.c_void_p(aligned), ctypes.byref(got),
                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "lbm_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls -------------------------------------------------------------------------
    def set_tiling(self, tx: int, ty: int, tz: int):
        _check(lib().lbm_set_tiling(self._h, tx, ty, tz), "lbm_set_tiling")
        return self

    def init(self, rho_r, rho_b=None, u=None, solid=None, pops=None):
        """Arrays may be torch tensors (device or host) or numpy arrays, FP64 (uint8 for
        solid), contiguous, node-ordered."""
        self._keep = (rho_r, rho_b, u, solid, pops)
        self._solid = solid
        self._has_walls = solid is not None
        _check(lib().lbm_init_fields(self._h, _ptr(rho_r), _ptr(rho_b), _ptr(u), _ptr(solid), _ptr(pops)),
               "lbm_init_fields")
        return self

    def step(self, nsteps: int = 1):
        fn = lib().lbm_step_cg if self.params.model == CG else lib().lbm_step_sc
        _check(fn(self._h, int(nsteps)), "lbm_step")
        return self

    def moments_into(self, rho_r=None, rho_b=None, u=None, pops=None, totals=None) -> int:
        """Raw lbm_moments into caller buffers; returns the status (OK or EUNSTABLE)."""
        rc = lib().lbm_moments(self._h, _ptr(rho_r), _ptr(rho_b), _ptr(u), _ptr(pops), _ptr(totals))
        if rc not in (OK, EUNSTABLE):
            raise LbmError(rc, "lbm_moments")
        return rc

    def moments(self, device: bool = True):
        """(rho_r, rho_b, u, totals-dict, status) with FP64 tensors on the device (or numpy)."""
        import torch
        p = self.params
        if device:
            rr = torch.empty(p.n, dtype=torch.float64, device=self.device)
            rb = torch.empty_like(rr)
            u = torch.empty(3, p.n, dtype=torch.float64, device=self.device)
        else:
            rr, rb, u = np.empty(p.n), np.empty(p.n), np.empty((3, p.n))
        t = np.zeros(NTOTALS)
        rc = self.moments_into(rr, rb, u, None, t)
        return rr, rb, u, dict(zip(TOTAL_NAMES, t.tolist())), rc

    def totals(self):
        t = np.zeros(NTOTALS)
        rc = self.moments_into(totals=t)
        return dict(zip(TOTAL_NAMES, t.tolist())), rc

    def state_planes(self, z0: int, nplanes: int, out=None):
        """Raw state of the planes [z0, z0 + nplanes) as a packed uint8 device tensor
        (lbm_get_state_planes; enqueued on the lattice's stream)."""
        import torch
        nb = int(lib().lbm_state_planes_bytes(self._h, nplanes))
        if out is None:
            out = torch.empty(nb, dtype=torch.uint8, device=self.device)
        _check(lib().lbm_get_state_planes(self._h, z0, nplanes, _ptr(out)), "lbm_get_state_planes")
        return out

    def set_state_planes(self, z0: int, nplanes: int, buf):
        """Write packed raw state (state_planes' layout) into the planes [z0, z0 + nplanes)."""
        _check(lib().lbm_set_state_planes(self._h, z0, nplanes, _ptr(buf)), "lbm_set_state_planes")
        return self

    def pops(self, device: bool = True):
        import torch
        p = self.params
        if device:
            out = torch.empty(p.ncomp, p.q, p.n, dtype=torch.float64, device=self.device)
        else:
            out = np.empty((p.ncomp, p.q, p.n))
        self.moments_into(pops=out)
        if device:
            self.stream.synchronize()
        return out

    def launch_count(self) -> int:
        return int(lib().lbm_launch_count(self._h))

    def state_bytes(self) -> int:
        return int(lib().lbm_state_bytes(self._h))

    def save_state(self, out=None):
        """Raw device state (bitwise checkpoint) into a uint8 tensor on the device."""
        import torch
        if out is None:
            out = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        rc = lib().lbm_save_state(self._h, _ptr(out))
        if rc not in (OK, EUNSTABLE):
            raise LbmError(rc, "lbm_save_state")
        return out

    def load_state(self, state, solid=None):
        self._keep_state = (state, solid)
        self._solid = solid
        self._has_walls = solid is not None
        _check(lib().lbm_load_state(self._h, _ptr(state), _ptr(solid)), "lbm_load_state")
        return self


class Batch:
    """Batched stepping of many lattices in one persistent launch per step (lbm_batch_*).
    The device job table is held as a torch tensor; all jobs must share the batch's stream
    and storage precision."""

    def __init__(self, precision: int, max_jobs: int, max_units: int, stream=None, device=None):
        import torch
        L = lib()
        need = ctypes.c_size_t(0)
        _check(L.lbm_batch_create(precision, max_jobs, max_units, None, ctypes.byref(need), None, None),
               "lbm_batch_create(size)")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.precision = precision
        self.ws = torch.empty(need.value + 256, dtype=torch.uint8, device=dev)
        aligned = (self.ws.data_ptr() + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        h = ctypes.c_void_p()
        got = ctypes.c_size_t(need.value)
        _check(L.lbm_batch_create(precision, max_jobs, max_units, ctypes.c_void_p(aligned), ctypes.byref(got),
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "lbm_batch_create")
        self._h = h
        self.jobs = []

    @staticmethod
    def units(lat: "Lattice") -> int:
        u = ctypes.c_int32(0)
        _check(lib().lbm_batch_units(lat._h, ctypes.byref(u)), "lbm_batch_units")
        return u.value

    def set(self, lattices, nsteps):
        n = len(lattices)
        hs = (_VP * max(n, 1))(*[lat._h for lat in lattices])
        st = (ctypes.c_int32 * max(n, 1))(*[int(k) for k in nsteps])
        _check(lib().lbm_batch_set(self._h, hs, st, n), "lbm_batch_set")
        self.jobs = list(lattices)  # keep the contexts alive while they are in the table
        return self

    def step(self, nsteps: int, graph: bool = True):
        _check(lib().lbm_batch_step(self._h, int(nsteps), int(bool(graph))), "lbm_batch_step")
        return self

    def launch_count(self) -> int:
        return int(lib().lbm_batch_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
