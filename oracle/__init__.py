"""FP64 CPU oracle of the two-component lattice Boltzmann step (arXiv 2110.05197, Sec. 2).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The product library never loads it
and shares no code with it (see ``lbm_oracle.c`` for the equations and their readings).

The C source is compiled by :func:`build` (plain gcc, OpenMP, contraction off) into
``liblbm_oracle.so`` beside it; :class:`OracleSim` wraps it with numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

D2Q9, D3Q19 = 0, 1
CG, SC_MP, SC_2C, SC_MR = 0, 1, 2, 3
NTOTALS = 10
TOTAL_NAMES = ("mass_r", "mass_b", "mom_x", "mom_y", "mom_z", "e_kin", "max_u", "nonfinite",
               "min_rho_r", "min_rho_b")


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (idempotent unless ``force``)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h")))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("model", ctypes.c_int32),
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
        ("Ga", ctypes.c_double * 2), ("Gr", ctypes.c_double * 2),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(_Params)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_init.argtypes = [ctypes.c_void_p, dp, dp, dp, ctypes.c_void_p, dp]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_get_pops.argtypes = [ctypes.c_void_p, dp]
        L.orc_moments.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.orc_force.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_get_threads.restype = ctypes.c_int
        L.orc_lattice_tables.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), dp, dp, dp, dp]
        L.orc_phi.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        L.orc_mr_vectors.argtypes = [ctypes.POINTER(ctypes.c_int), dp]
        L.orc_mr_vectors.restype = ctypes.c_int
        L.orc_cg_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp,
                                         ctypes.c_double, ctypes.c_int, dp]
        L.orc_sc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_guo_source.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
        L.orc_perturbation.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_recolor.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, dp, ctypes.c_double,
                                  ctypes.c_double, dp, dp]
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def mr_vectors():
    """The 93 vectors of belts 1 and 2 and their weights p (Eq. pweights), as the oracle
    uses them: (c [93, 3] int, p [93])."""
    c = np.zeros(93 * 3, dtype=np.int32)
    p = np.zeros(93)
    m = lib().orc_mr_vectors(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(p))
    return c.reshape(-1, 3)[:m], p[:m]


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def q_of(lattice: int) -> int:
    return 9 if lattice == D2Q9 else 19


def lattice_tables(lattice: int):
    """(c [Q,3] int, w, B, psi, xi) as the oracle holds them."""
    q = ctypes.c_int()
    c = (ctypes.c_int * 57)()
    w, B, psi, xi = (np.zeros(19) for _ in range(4))
    lib().orc_lattice_tables(lattice, ctypes.byref(q), c, _p(w), _p(B), _p(psi), _p(xi))
    Q = q.value
    cc = np.array(list(c)[: 3 * Q], dtype=np.int64).reshape(Q, 3)
    return cc, w[:Q].copy(), B[:Q].copy(), psi[:Q].copy(), xi[:Q].copy()


def phi(lattice: int, alpha: float) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_phi(lattice, alpha, _p(out))
    return out[: q_of(lattice)].copy()


def cg_equilibrium(lattice, rho_k, alpha_k, u, grad_k, nubar, enhanced=1):
    out = np.zeros(19)
    lib().orc_cg_equilibrium(lattice, rho_k, alpha_k, _p(_f64(u)), _p(_f64(grad_k)), nubar,
                             int(enhanced), _p(out))
    return out[: q_of(lattice)].copy()


def sc_equilibrium(lattice, rho, u):
    out = np.zeros(19)
    lib().orc_sc_equilibrium(lattice, rho, _p(_f64(u)), _p(out))
    return out[: q_of(lattice)].copy()


def guo_source(lattice, u, F, omega):
    out = np.zeros(19)
    lib().orc_guo_source(lattice, _p(_f64(u)), _p(_f64(F)), omega, _p(out))
    return out[: q_of(lattice)].copy()


def perturbation(lattice, grad_n, A, eps=0.0):
    out = np.zeros(19)
    lib().orc_perturbation(lattice, _p(_f64(grad_n)), A, eps, _p(out))
    return out[: q_of(lattice)].copy()


def recolor(lattice, fstar, rho_r, rho_b, alpha_r, alpha_b, grad_n, beta, eps=0.0):
    fr, fb = np.zeros(19), np.zeros(19)
    fs = np.zeros(19)
    fs[: q_of(lattice)] = fstar
    lib().orc_recolor(lattice, _p(fs), rho_r, rho_b, alpha_r, alpha_b, _p(_f64(grad_n)), beta,
                      eps, _p(fr), _p(fb))
    Q = q_of(lattice)
    return fr[:Q].copy(), fb[:Q].copy()


@dataclass
class Params:
    """Mirror of ``orc_params``; defaults follow the paper where it gives a value."""
    lattice: int = D3Q19
    model: int = CG
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
    Ga: tuple = (0.0, 0.0)       # SC_MR: attractive self-couplings G^a of species A, B
    Gr: tuple = (0.0, 0.0)       # SC_MR: repulsive self-couplings G^r of species A, B

    def to_c(self) -> _Params:
        p = _Params()
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
        return q_of(self.lattice)

    @property
    def ncomp(self) -> int:
        return 1 if self.model == SC_MP else 2

    @property
    def alpha_r(self) -> float:
        return 1.0 - (1.0 - self.alpha_b) * self.rho_b0 / self.rho_r0


class OracleSim:
    """One simulation held by the oracle.  Arrays are node-ordered (x fastest)."""

    def __init__(self, params: Params):
        self.params = params
        self._cp = params.to_c()
        self._h = lib().orc_create(ctypes.byref(self._cp))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho_r, rho_b=None, u=None, solid=None, pops=None):
        rr = _f64(np.asarray(rho_r).reshape(-1))
        rb = _f64(np.zeros_like(rr) if rho_b is None else np.asarray(rho_b).reshape(-1))
        uu = None if u is None else _f64(np.asarray(u).reshape(3, -1))
        so = None
        if solid is not None:
            so = np.ascontiguousarray(np.asarray(solid).reshape(-1), dtype=np.uint8)
        pp = None if pops is None else _f64(np.asarray(pops).reshape(-1))
        self._keep = (rr, rb, uu, so, pp)
        rc = lib().orc_init(self._h, _p(rr), _p(rb), _p(uu),
                            None if so is None else so.ctypes.data_as(ctypes.c_void_p), _p(pp))
        if rc:
            raise RuntimeError("orc_init failed")
        return self

    def step(self, nsteps: int = 1):
        if lib().orc_step(self._h, int(nsteps)):
            raise RuntimeError("orc_step failed")
        return self

    def pops(self) -> np.ndarray:
        p = self.params
        out = np.zeros((p.ncomp, p.q, p.n))
        lib().orc_get_pops(self._h, _p(out))
        return out

    def moments(self):
        p = self.params
        rr, rb, u, t = np.zeros(p.n), np.zeros(p.n), np.zeros((3, p.n)), np.zeros(NTOTALS)
        lib().orc_moments(self._h, _p(rr), _p(rb), _p(u), _p(t))
        return rr, rb, u, t

    def totals(self) -> dict:
        return dict(zip(TOTAL_NAMES, self.moments()[3]))

    def force(self) -> np.ndarray:
        out = np.zeros((3, self.params.n))
        lib().orc_force(self._h, _p(out))
        return out
