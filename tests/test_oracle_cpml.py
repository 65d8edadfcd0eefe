"""Pins of the oracle's CPML absorbing layers (Sec. 3.2) and of the laser
current sheet that goes with them, against what the mathematics fixes:

* with sigma = alpha = 0 and kappa = 1 the layers do nothing and the box is a
  perfect-conductor cavity: a standing mode sin(k x) oscillates at the
  discrete Yee frequency sin(omega dt / 2) = (dt / dx) sin(k dx / 2);
* a wave packet at normal incidence leaves less than 1e-8 of its energy
  behind,
  and fields travelling in every direction decay, while the same run
  without loss keeps its energy;
* the current sheet launches a wave of the prescribed amplitude into +x and
  the wave it sends into -x is absorbed.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _fields_step(g, t):
    O.maxwell_half(g, 0, t)
    O.maxwell_half(g, 1, t + 0.5 * g.dt)


def _field_energy(g):
    return sum(0.5 * (np.sum(g.E[c] ** 2) + np.sum(g.B[c] ** 2)) for c in range(3)) * g.dV


def test_lossless_layers_are_a_conducting_cavity():
    nx, ny, dx = 64, 4, 0.1
    dt = 0.95 * dx / math.sqrt(2.0)
    g = O.Grid(2, (nx, ny), (dx, dx), dt, 1, absorb_x=True,
               pml=O.Pml(cells=8, sigma_max=0.0, kappa_max=1.0, alpha_max=0.0))
    m = 3
    k = m * math.pi / (nx * dx)
    x = np.arange(nx + 1) * dx
    g.E[2][0, :, :] = np.sin(k * x)[None, :]          # E_z at nodes, zero at both walls
    g.E[2][0, :, 0] = 0.0
    g.E[2][0, :, nx] = 0.0
    omega = 2.0 / dt * math.asin(dt / dx * math.sin(0.5 * k * dx))
    probe = nx // (2 * m)                               # an antinode
    steps = 200
    for s in range(steps):
        _fields_step(g, s * dt)
    got = g.E[2][0, 0, probe] / math.sin(k * x[probe])
    assert abs(got - math.cos(omega * steps * dt)) < 1e-10
    assert np.all(g.E[2][0, :, 0] == 0.0) and np.all(g.E[2][0, :, nx] == 0.0)


def _packet(g, x0, w, k0):
    """E_z, B_y of a wave packet travelling in +x (B_y = -E_z at the staggered
    point, half a step earlier)."""
    nx = g.nx
    f = lambda x: np.exp(-((x - x0) / w) ** 2) * np.sin(k0 * (x - x0))
    x_n = np.arange(nx + 1) * g.dx
    x_h = (np.arange(nx + 1) + 0.5) * g.dx
    g.E[2][0, :, :] = f(x_n)[None, :]
    g.E[2][0, :, 0] = 0.0
    g.E[2][0, :, nx] = 0.0
    by = -f(x_h + 0.5 * g.dt)
    by[-1] = 0.0
    g.B[1][0, :, :] = by[None, :]


@pytest.mark.parametrize("alpha_max", [0.0, 0.05])
def test_normal_incidence_packet_is_absorbed(alpha_max):
    nx, ny, dx = 400, 4, 0.1
    dt = 0.95 * dx / math.sqrt(2.0)
    g = O.Grid(2, (nx, ny), (dx, dx), dt, 1, absorb_x=True, pml=O.Pml(cells=16, alpha_max=alpha_max))
    _packet(g, 0.5 * nx * dx, 2.0, 2.0 * math.pi / (20 * dx))
    e0 = _field_energy(g)
    for s in range(int(1.0 * nx * dx / dt)):           # out and a reflection would be back
        _fields_step(g, s * dt)
    assert _field_energy(g) < 1e-8 * e0


@pytest.mark.parametrize("lossy", [False, True])
def test_fields_in_all_directions_decay(lossy):
    nx, ny, dx = 96, 48, 0.1
    dt = 0.95 * dx / math.sqrt(2.0)
    pml = O.Pml(cells=16) if lossy else O.Pml(cells=16, sigma_max=0.0, alpha_max=0.0)
    g = O.Grid(2, (nx, ny), (dx, dx), dt, 1, absorb_x=True, pml=pml)
    rng = np.random.Generator(np.random.Philox(4))
    # a smooth random E_z in the middle of the box: plane waves within 60
    # degrees of the x axis (either way; waves along y never reach an x
    # layer in a box periodic in y), wavelengths of 12 cells or more, under a
    # window
    xi = np.arange(nx + 1)[None, :] * dx
    yi = (np.arange(ny)[:, None] + 0.5) * dx
    f = np.zeros((ny, nx + 1))
    for _ in range(24):
        th = rng.uniform(-math.pi / 3, math.pi / 3) + math.pi * rng.integers(0, 2)
        kmag = 2.0 * math.pi / (dx * rng.uniform(12.0, 30.0))
        ky = 2.0 * math.pi * round(kmag * math.sin(th) * ny * dx / (2.0 * math.pi)) / (ny * dx)
        f += rng.standard_normal() * np.cos(kmag * math.cos(th) * xi + ky * yi + rng.uniform(0, 6.3))
    f *= np.exp(-((np.arange(nx + 1) - nx / 2) / 12.0) ** 2)[None, :]
    g.E[2][0] = f
    g.E[2][0, :, 0] = 0.0
    g.E[2][0, :, nx] = 0.0
    e0 = _field_energy(g)
    steps = int(4.0 * nx * dx / dt)
    for s in range(steps):
        _fields_step(g, s * dt)
    e1 = _field_energy(g)
    if lossy:
        assert e1 < 1e-2 * e0           # measured 4e-3 (waves near 60 degrees leave slowly)
    else:
        assert abs(e1 / e0 - 1.0) < 0.03      # a closed cavity keeps its energy (up to the E/B staggering)


def test_laser_sheet_amplitude_and_direction():
    nx, ny, dx = 400, 8, 2 * math.pi / 32
    dt = 0.95 * dx / math.sqrt(2.0)
    a0, tau = 1.0, 4 * 2 * math.pi
    laser = O.Laser(a0, 1e6, tau, 1.0, 0.5 * ny * dx, 0.0)      # plane wave (huge waist)
    g = O.Grid(2, (nx, ny), (dx, dx), dt, 1, absorb_x=True, laser=laser, pml=O.Pml(cells=16))
    probe = 200
    peak, left = 0.0, 0.0
    steps = int((tau + (probe - 18) * dx) / dt) + 40
    for s in range(steps):
        _fields_step(g, s * dt)
        peak = max(peak, float(np.max(np.abs(g.E[1][0, :, probe]))))
    # the largest value of a0 sin^2(pi s / tau) sin(s) (the carrier's crests
    # miss the envelope's top), within the grid dispersion
    ss = np.linspace(0.0, tau, 200001)
    expect = a0 * np.max(np.abs(np.sin(np.pi * ss / tau) ** 2 * np.sin(ss)))
    assert abs(peak / expect - 1.0) < 0.02
    # behind the sheet (between the layer and the sheet) nothing is left once the
    # pulse has been emitted, and the backward half was absorbed by the layer
    tail = g.E[1][0, :, 0:17]
    assert float(np.max(np.abs(tail))) < 1e-3 * a0
