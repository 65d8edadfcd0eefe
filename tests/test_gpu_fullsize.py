"""Long runs and the full-size benchmark workload.

* The plain 2D thermal plasma (64 x 64, 16 per cell, CIC) for its full 200
  steps: the total-energy history of the GPU paths follows the oracle's
  within 1 % of the initial energy at every sample (PIC is chaotic, so long
  runs are compared on histories, not element by element).
* The 2D laser-plasma at full size (2048 x 1024, 67 M particles, TSC, FP32
  fixed point): a random sample of particles pushed by the oracle in the
  GPU's own fields agrees with the GPU push to float32 precision, and the
  integer continuity identity holds exactly on the whole grid.  The same
  check at full size for the 3D thermal plasma (256^3, TSC), the 3D
  laser-target (512 x 256^2, CIC, laser on the slab) and one member of the
  96-member ensemble stepped through the batched path.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_13507_b300 import workloads as W

from pic_cases import gpu_case, oracle_case, sampled_push_check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13507_b300 import build, lpic
    build.build()
    lpic.load()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_history_200_steps(precision):
    from paper_2607_13507_b300 import lpic
    wl = W.thermal2d()                       # 64 x 64, 16 per cell, 200 steps
    parts = W.load_all(wl)
    g, sps = oracle_case(wl, parts)
    G = gpu_case(wl, parts, lpic.FP64 if precision == "fp64" else lpic.FP32_FIXED)
    e0 = None
    hist_g, hist_o = [], []
    for s in range(wl.steps + 1):
        if s % 10 == 0:
            torch.cuda.synchronize()
            d = G.diagnostics()
            ek, ef, _ = O.energy(g, sps)
            hist_g.append(d.kinetic + d.field)
            hist_o.append(ek + ef)
            if e0 is None:
                e0 = ek + ef
        if s < wl.steps:
            O.step(g, sps, s * wl.dt)
            G.step(s * wl.dt)
    hist_g, hist_o = np.array(hist_g), np.array(hist_o)
    assert np.max(np.abs(hist_g - hist_o)) < 0.01 * e0
    # the heating itself (finite-grid instability at dx = 10 Debye lengths)
    # must be reproduced, not just the initial energy
    dg, do = hist_g - hist_g[0], hist_o - hist_o[0]
    assert np.max(np.abs(dg - do)) < 0.01 * max(np.max(np.abs(do)), 1e-3 * e0)
    assert G.check_status() == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_heating_setup_energy_history(precision):
    """The numerical-heating set-up (n_e = 10 n_c, 1 keV Maxwell-Juttner
    electrons and ions, CIC, periodic) on a 32 x 32 box at dx = lambda/20,
    16 particles per cell and species: 300 steps, total energy within 1 % of
    the initial energy of the oracle's at every 10th step, and the drift
    itself reproduced to 1 %."""
    from paper_2607_13507_b300 import lpic
    wl = W.heating2d(res=20, ppc=16, L_lambda=1.6)
    parts = W.load_all(wl)
    g, sps = oracle_case(wl, parts)
    G = gpu_case(wl, parts, lpic.FP64 if precision == "fp64" else lpic.FP32_FIXED)
    hist_g, hist_o = [], []
    for s in range(301):
        if s % 10 == 0:
            torch.cuda.synchronize()
            d = G.diagnostics()
            ek, ef, _ = O.energy(g, sps)
            hist_g.append(d.kinetic + d.field)
            hist_o.append(ek + ef)
        if s < 300:
            O.step(g, sps, s * wl.dt)
            G.step(s * wl.dt)
    hist_g, hist_o = np.array(hist_g), np.array(hist_o)
    e0 = hist_o[0]
    assert np.max(np.abs(hist_g - hist_o)) < 0.01 * e0
    dg, do = hist_g - hist_g[0], hist_o - hist_o[0]
    assert np.max(np.abs(dg - do)) < 0.01 * max(np.max(np.abs(do)), 1e-3 * e0)
    assert G.check_status() == 0


def test_laser2d_full_size_sampled_push_and_exact_continuity():
    from paper_2607_13507_b300 import lpic
    wl = W.laser2d()
    parts = W.load_all(wl)
    G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=(16, 8), block_particles=8192)
    for p in parts:
        G.add_species(p)
    del parts
    for s in range(3):
        G.step(s * wl.dt)
    # state at the start of step 3: fields after its first half step
    t3 = 3 * wl.dt
    G.maxwell_half(0, t3)
    G.zero_current()
    sp = G.species[0]
    G.sort(sp.id)
    st = sp.state()
    rng = np.random.Generator(np.random.Philox(5))
    pick = rng.choice(st["id"].shape[0], size=2000, replace=False)
    ids = st["id"][pick]
    rho0 = sp.charge()
    # the oracle push of the sample in the GPU's fields
    g = O.Grid(2, wl.n, wl.h, wl.dt, wl.order, absorb_x=True)
    for c in range(3):
        g.E[c][...] = G.E[c].cpu().numpy().astype(np.float64)
        g.B[c][...] = G.B[c].cpu().numpy().astype(np.float64)
    h = np.array(wl.h)[:, None]
    u = st["u"][:, pick].astype(np.float64)
    gam = np.sqrt(1.0 + (u ** 2).sum(0))
    xh = (st["cell"][pick] % wl.n[0], st["cell"][pick] // wl.n[0])
    x_half = (np.stack(xh).astype(np.float64) + st["off"][:, pick].astype(np.float64)) * h
    x_int = x_half - 0.5 * wl.dt * u[:2] / gam
    osp = O.Species(-1.0, 1.0, x_int, u, st["w"][pick].astype(np.float64))
    O.push_species(g, osp)
    # the GPU push of all particles
    G.gather_push_deposit(sp.id)
    torch.cuda.synchronize()
    assert G.check_status() == 0
    st1 = sp.state()
    x1 = sp.positions_at_step()
    order = np.argsort(st1["id"])
    rows = order[np.searchsorted(st1["id"][order], ids)]
    assert np.array_equal(st1["id"][rows], ids)
    ug = st1["u"][:, rows].astype(np.float64)
    rel = np.linalg.norm(ug - osp.u) / np.linalg.norm(osp.u)
    assert rel < 1e-5, rel
    diff = x1[:, rows] - osp.x[:2]
    Ly = wl.n[1] * wl.h[1]
    diff[1] = np.remainder(diff[1] + 0.5 * Ly, Ly) - 0.5 * Ly      # periodic y
    dx = np.abs(diff) / h
    assert np.max(dx) < 1e-5, np.max(dx)
    # exact integer continuity over the whole grid (absorbing x: interior columns)
    rho1 = sp.charge()
    J = G.J
    div = (J[0] - torch.roll(J[0], 1, 2)) + (J[1] - torch.roll(J[1], 1, 1))
    res = (rho1 - rho0 + div)[:, :, 4:-4]
    assert torch.count_nonzero(res).item() == 0


def test_thermal3d_full_size_sampled_push_and_exact_continuity():
    """The 3D roofline workload at its full size (256^3, TSC, 134 M
    particles, 8x8x4 tiles of 4096 particles per block): after three steps,
    2000 particles drawn at random are pushed by the oracle in the GPU's own
    fields (momenta <= 1e-5 relative, positions <= 1e-5 cell), and the
    integer continuity of the step holds exactly on every node."""
    from paper_2607_13507_b300 import lpic
    wl = W.thermal3d()
    parts = W.load_all(wl)
    G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=(8, 8, 4), block_particles=4096)
    G.add_species(parts[0])
    del parts
    for s in range(3):
        G.step(s * wl.dt)
    rel_u, dx, nonzero = sampled_push_check(G, wl, G.species[0], 3 * wl.dt)
    assert rel_u < 1e-5, rel_u
    assert dx < 1e-5, dx
    assert nonzero == 0


def test_laser3d_full_size_sampled_push_and_exact_continuity():
    """The 3D laser-target workload at its full size (512x256^2, CIC, 134 M
    particles, slab tiles crowded next to empty vacuum tiles) after 400
    steps, with the laser on the slab: electrons and protons each checked on
    2000 particles against the oracle and by exact integer continuity."""
    from paper_2607_13507_b300 import lpic
    wl = W.laser3d()
    parts = W.load_all(wl)
    G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=(8, 8, 4), block_particles=8192)
    for p in parts:
        G.add_species(p)
    del parts
    steps = 400
    for s in range(steps):
        G.step(s * wl.dt)
    torch.cuda.synchronize()
    assert G.check_status() == 0
    t = steps * wl.dt
    for k, sp in enumerate(G.species):
        rel_u, dx, nonzero = sampled_push_check(G, wl, sp, t, seed=7 + k)
        assert rel_u < 1e-5, (k, rel_u)
        assert dx < 1e-5, (k, dx)
        assert nonzero == 0, k
        # the next species starts a fresh step on the same fields
        G.maxwell_half(1, t + 0.5 * wl.dt)
        t += wl.dt


def test_ensemble_member_full_size_sampled_push_and_exact_continuity():
    """The 96-member batched ensemble (sides 128-768, 4-64 particles per cell,
    one persistent particle kernel over the device queue, replayed graphs):
    after three ensemble steps, member 0 is checked like the single grids."""
    from paper_2607_13507_b300 import lpic
    members = W.ensemble()
    grids = []
    for wl in members:
        G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=(16, 8))
        G.add_species(W.load_all(wl)[0])
        grids.append(G)
    ens = lpic.Ensemble(grids)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    ens.graph_steps(3, side)
    torch.cuda.synchronize()
    assert ens.check_status(side) == 0
    ens.close()
    wl, G = members[0], grids[0]
    rel_u, dx, nonzero = sampled_push_check(G, wl, G.species[0], 3 * wl.dt)
    assert rel_u < 1e-5, rel_u
    assert dx < 1e-5, dx
    assert nonzero == 0
