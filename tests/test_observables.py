"""The host-side observable measurements (tests/observables.py) on fields with known
answers, so that the precision comparisons in test_gpu_observables.py measure what they
say."""
import numpy as np
import pytest

from tests import observables as obs

pytest.importorskip("scipy")


def test_frequency_of_a_damped_cosine():
    dt, w = 20.0, 5.3e-3
    t = np.arange(1, 121) * dt
    r = 12.0 + 0.8 * np.exp(-1e-3 * t) * np.cos(w * t + 0.3) + 1e-4 * t / t[-1]
    assert abs(obs.oscillation_frequency(r, dt) - w) / w < 1e-3


def test_radius_along_x_of_a_sphere():
    n, R = 40, 9.3
    x = np.arange(n) - (n - 1) / 2
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    d = np.sqrt(xx ** 2 + y ** 2 + z ** 2)
    # smooth interface: rho^N = tanh((R - d)/2) with rho_r + rho_b = 1
    col = np.tanh((R - d) / 2.0).ravel()
    rr, rb = (1 + col) / 2, (1 - col) / 2
    # the x line through the box centre sits half a node off the sphere's centre in y and z
    off = np.sqrt(2 * 0.5 ** 2)
    assert abs(obs.radius_along_x(rr, rb, (n, n, n)) - np.sqrt(R ** 2 - off ** 2)) < 0.05


def test_pressure_jump_of_a_step():
    col = np.where(np.arange(100) < 40, 1.0, -1.0)
    rr = np.where(col > 0, 1.02, 0.0)
    rb = np.where(col > 0, 0.0, 0.1)
    assert obs.pressure_jump(rr, rb, 0.4, 0.3) == pytest.approx(0.4 * 1.02 - 0.3 * 0.1)


def test_components_join_across_periodic_faces():
    shape = (4, 6, 10)
    m = np.zeros(shape, bool)
    m[1:3, 2:4, 0:2] = True
    m[1:3, 2:4, 8:10] = True      # the same drop through the x face
    m[0, 0, 5] = True
    m[3, 0, 5] = True             # joined through the z face
    lab = obs.periodic_components(m)
    assert len(np.unique(lab[lab > 0])) == 2
    rr = np.where(m, 1.0, 0.0).ravel()
    rb = np.where(m, 0.0, 1.0).ravel()
    assert obs.droplet_masses(rr, rb, shape) == [16.0, 2.0]


def test_endpoint_along_z_of_a_capsule():
    nx = ny = 16
    nz = 64
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx = cy = (nx - 1) / 2
    cz = (nz - 1) / 2
    half = 12.0                     # cylinder half-length; caps of radius 4 beyond it
    dz = np.clip(np.abs(z - cz) - half, 0.0, None)
    d = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + dz ** 2)
    col = np.tanh((4.0 - d) / 2.0).ravel()
    rr, rb = (1 + col) / 2, (1 - col) / 2
    # the z line through (nx // 2, ny // 2) sits 0.5 off the axis in x and y
    tip = half + np.sqrt(4.0 ** 2 - 2 * 0.5 ** 2)
    assert abs(obs.endpoint_along_z(rr, rb, (nz, ny, nx)) - tip) < 0.05
