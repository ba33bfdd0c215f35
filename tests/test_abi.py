"""The C-ABI library builds, loads and exports every entry point include/*.h declares; the
size query and argument validation work without a GPU (no compute calls here)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2110_05197_gb300 import build as lbm_build
from paper_2110_05197_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    lbm_build.build()
    return lbm.lib()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lbm_create", "lbm_init_fields", "lbm_step_cg", "lbm_step_sc", "lbm_moments",
                     "lbm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    names = _declared_functions()
    assert names
    for n in names:
        assert hasattr(L, n), n
        assert n in lbm.SIGNATURES, f"binding lacks {n}"


def _size(L, **kw):
    p = lbm.Params(**kw).to_c()
    need = ctypes.c_size_t(0)
    rc = L.lbm_create(ctypes.byref(p), None, ctypes.byref(need), None, None)
    return rc, need.value


def test_workspace_size_query(L):
    rc, b = _size(L, nx=128, ny=128, nz=128, precision=lbm.FP32, model=lbm.CG)
    assert rc == lbm.OK
    N = 128 ** 3
    pops = 2 * 2 * 19 * N * 4   # A/B populations
    ref = 2 * 2 * N * 4         # A/B reference densities
    # + FP64 staging for moments (rho_r, rho_b, u, psi: 6 N doubles), wall mask, partials
    assert pops + ref < b < pops + ref + 6 * N * 8 + 2 * N + (1 << 20)
    rc, b64 = _size(L, nx=128, ny=128, nz=128, precision=lbm.FP64, model=lbm.CG)
    assert b64 - b == 2 * 2 * 19 * N * 4 + ref
    rc, b16 = _size(L, nx=128, ny=128, nz=128, precision=lbm.FP16, model=lbm.CG)
    assert b - b16 == 2 * 2 * 19 * N * 2
    rc, bsc = _size(L, nx=128, ny=128, nz=128, precision=lbm.FP32, model=lbm.SC_MP)
    assert b - bsc == 2 * 19 * N * 4 + 2 * N * 4
    # in-place streaming keeps one population buffer and one reference field
    rc, baa = _size(L, nx=128, ny=128, nz=128, precision=lbm.FP32, model=lbm.CG, streaming=lbm.STREAM_AA)
    assert rc == lbm.OK and b - baa == (pops + ref) // 2


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(lattice=lbm.D2Q9, nz=4), dict(tau_r=0.5), dict(precision=4), dict(model=9),
    dict(rho_b0=-1.0), dict(model=lbm.SC_MP, rho0_psi=0.0), dict(diag_every=-1),
    dict(rho_r0=0.1, rho_b0=1.0),  # alpha_R < 0 from Eq. gamma
    dict(streaming=2),
    dict(model=lbm.SC_MR, lattice=lbm.D2Q9, nz=1), dict(model=4),
])
def test_invalid_parameters_rejected(L, bad):
    rc, _ = _size(L, **bad)
    assert rc == lbm.EINVAL


def test_status_strings(L):
    for s in range(7):
        assert L.lbm_status_string(s)
    assert L.lbm_destroy(None) == lbm.OK
    assert L.lbm_launch_count(None) == 0
    assert L.lbm_step_cg(None, 1) == lbm.EINVAL
    assert L.lbm_moments(None, None, None, None, None, None) == lbm.EINVAL


def test_sweep_trace_is_seeded_and_in_range():
    """The serving sweep's request trace (host only): seeded, parameters in the stated
    ranges, arrivals increasing."""
    from paper_2110_05197_gb300 import serve
    a = serve.sweep(64, seed=5, steps=(5000, 20000), rate_hz=2.0)
    b = serve.sweep(64, seed=5, steps=(5000, 20000), rate_hz=2.0)
    assert [(r.grid, r.model, r.steps, r.kw) for r in a] == [(r.grid, r.model, r.steps, r.kw) for r in b]
    assert all(x.arrival < y.arrival for x, y in zip(a, a[1:]))
    for r in a:
        assert r.grid in serve.GRIDS and 5000 <= r.steps <= 20000
        if r.model == lbm.CG:
            assert 1e-3 <= r.kw["rho_b0"] <= 1.0 and 1e-4 <= r.kw["A"] <= 1e-1
            assert 0.5 < r.kw["tau_r"] <= 3 * 10 / 6 + 0.5
        else:
            assert 4.2 <= -r.kw["G"] <= 6.5
    assert {r.model for r in a} == {lbm.CG, lbm.SC_MP}


def test_tuner_candidates():
    from paper_2110_05197_gb300 import tune
    c = tune.candidates_for(lbm.Params(nx=128, ny=128, nz=128))
    assert (32, 8, 0) in c and (64, 4, 0) in c and (32, 4, 0) in c
    # the field-pass kernels (in-place streaming, multirange model) pick their own shape
    assert tune.candidates_for(lbm.Params(nx=64, ny=64, nz=64, streaming=lbm.STREAM_AA)) == [(32, 8, 0)]
    assert tune.candidates_for(lbm.Params(nx=64, ny=64, nz=64, model=lbm.SC_MR)) == [(32, 8, 0)]


def test_multirange_workspace_and_limits(L):
    rc, b = _size(L, nx=64, ny=64, nz=64, model=lbm.SC_MR, precision=lbm.FP32)
    rc2, b2 = _size(L, nx=64, ny=64, nz=64, model=lbm.SC_2C, precision=lbm.FP32)
    assert rc == rc2 == lbm.OK and b == b2      # same storage as the two-component model
    rc, _ = _size(L, nx=1, ny=64, nz=64, model=lbm.SC_MR)
    assert rc == lbm.EINVAL                     # the repulsion reaches two nodes


def test_noalloc_binding_refuses_host_buffers(L):
    """The binding checks what the C entry point cannot (it receives raw pointers): a host
    tensor or array is refused before any call, on any machine."""
    torch = pytest.importorskip("torch")
    p = lbm.Params(nx=4, ny=4, nz=4)
    for pops in (torch.zeros(2 * 19 * p.n, dtype=torch.float64), np.zeros(2 * 19 * p.n)):
        with pytest.raises(lbm.LbmError) as e:
            lbm.totals_noalloc(p, pops)
        assert e.value.status == lbm.EINVAL
