"""Edge cases of the CUDA path: an empty species, particles at rest and on
cell boundaries, a crowded cell split over several work items, the smallest
grid (4 cells a side, smaller than a tile) -- each against the oracle or an
exact property."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_13507_b300 import workloads as W

from pic_cases import gpu_case, match_particles, oracle_case, rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13507_b300 import build, lpic
    build.build()
    lpic.load()


def _particles(dim, cells, offs, us, w=0.01, q=-1.0, m=1.0):
    n = len(cells)
    return W.Particles(q, m, np.array(cells, dtype=np.int32).T.reshape(dim, n),
                       np.array(offs, dtype=np.float32).T.reshape(dim, n),
                       np.array(us, dtype=np.float32).T.reshape(3, n),
                       np.full(n, w, dtype=np.float32), np.arange(n, dtype=np.int32))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_empty_species_changes_nothing(precision):
    from paper_2607_13507_b300 import lpic
    prec = lpic.FP64 if precision == "fp64" else lpic.FP32_FIXED
    wl = W.thermal2d(n=24, ppc=4, vth=0.1, order=2, precision=precision)
    parts = W.load_all(wl)
    empty = W.Particles(1.0, 1836.0, np.zeros((2, 0), np.int32), np.zeros((2, 0), np.float32),
                        np.zeros((3, 0), np.float32), np.zeros(0, np.float32), np.zeros(0, np.int32))
    A = gpu_case(wl, parts, prec)
    B = gpu_case(wl, [empty] + parts, prec)
    for s in range(4):
        A.step(s * wl.dt)
        B.step(s * wl.dt)
    torch.cuda.synchronize()
    assert A.check_status() == 0 and B.check_status() == 0
    assert B.species[0].query()[1] == 0
    tol = 0.0 if precision == "fp32" else 1e-13      # FP64 atomics add in any order
    for c in range(3):
        for a, b in ((A.E[c], B.E[c]), (A.B[c], B.B[c])):
            d = float((a - b).abs().max())
            assert d <= tol * max(float(a.abs().max()), 1e-300)


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 2)])
def test_particles_at_rest_on_cell_faces(dim, order):
    """Offsets 0 and just below 1, zero momentum, no fields: the current is
    exactly zero and nothing moves; FP32 continuity holds."""
    from paper_2607_13507_b300 import lpic
    if dim == 2:
        wl = W.thermal2d(n=8, ppc=1, vth=0.0, order=order, precision="fp32")
    else:
        wl = W.thermal3d(n=8, ppc=1, vth=0.0, order=order, precision="fp32")
    below1 = float(np.nextafter(np.float32(1.0), np.float32(0.0)))
    cells, offs = [], []
    for k, o in enumerate([0.0, below1, 0.5, 0.25]):
        cells.append([3 + k % 2] * dim)
        offs.append([o] * dim)
    p = _particles(dim, cells, offs, [[0.0, 0.0, 0.0]] * len(cells))
    G = gpu_case(wl, [p], lpic.FP32_FIXED)
    for s in range(3):
        G.step(s * wl.dt)
    torch.cuda.synchronize()
    assert G.check_status() == 0
    for c in range(3):
        assert int(G.J[c].abs().max()) == 0
    st = G.species[0].state()
    o = np.argsort(st["id"])
    assert np.array_equal(st["off"][:, o], p.off)


@pytest.mark.parametrize("dim", [2, 3])
def test_crowded_cell_over_several_work_items(dim):
    """8193 particles in one cell with 8192 particles per work item: two items
    of one tile add their currents; against the oracle and exact continuity."""
    from paper_2607_13507_b300 import lpic
    if dim == 2:
        wl = W.thermal2d(n=16, ppc=1, vth=0.0, order=2, precision="fp32")
    else:
        wl = W.thermal3d(n=8, ppc=1, vth=0.0, order=2, precision="fp32")
    n = 8193
    rng = np.random.Generator(np.random.Philox(9))
    cells = [[4] * dim] * n
    offs = rng.random((n, dim), dtype=np.float32)
    us = (0.2 * rng.standard_normal((n, 3))).astype(np.float32)
    p = _particles(dim, cells, offs, us, w=1e-4)
    g, sps = oracle_case(wl, [p])
    G = lpic.grid_for(wl, lpic.FP32_FIXED, block_particles=8192)
    G.add_species(p)
    rho0 = G.species[0].charge()
    run_oracle(g, sps, 2)
    run_gpu(G, 2)
    assert G.check_status() == 0
    Jg = G.current()
    for c in range(3):
        assert rel_l2(Jg[c].cpu().numpy(), g.J[c]) < 3e-4
    xg, xo, ug, uo = match_particles(G, G.species[0], sps[0], wl)
    assert rel_l2(ug, uo) < 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_smallest_grid_smaller_than_a_tile(precision):
    from paper_2607_13507_b300 import lpic
    wl = W.thermal2d(n=4, ppc=8, vth=0.1, order=2, precision=precision)
    parts = W.load_all(wl)
    g, sps = oracle_case(wl, parts)
    G = gpu_case(wl, parts, lpic.FP64 if precision == "fp64" else lpic.FP32_FIXED)
    run_oracle(g, sps, 5)
    run_gpu(G, 5)
    assert G.check_status() == 0
    tol = 1e-11 if precision == "fp64" else 5e-4
    for c in range(3):
        if np.linalg.norm(g.E[c]) > 0:
            assert rel_l2(G.E[c].cpu().numpy(), g.E[c]) < tol


def test_particle_outside_its_tile_sets_halo_status_in_the_unfused_stage():
    """The unfused stages run on freshly sorted particles, without a
    global-memory path: a particle that a caller moved out of its tile's box
    after the sort is skipped and raises LPIC_ST_HALO (made on the host: one
    cell index rewritten in the buffer, a valid cell of the grid)."""
    from paper_2607_13507_b300 import lpic
    wl = W.thermal2d(n=64, ppc=2, vth=0.05, order=2, precision="fp32")
    G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=(16, 16))
    sp = G.add_species(W.load_all(wl)[0])
    G.sort(sp.id)
    torch.cuda.synchronize()
    cur, n = sp.query()
    cells = sp._views(cur)["cell"]
    c0 = int(cells[0].item())
    x, y = c0 % 64, c0 // 64
    cells[0] = ((y + 32) % 64) * 64 + (x + 32) % 64          # two tiles away in x and y
    torch.cuda.synchronize()
    G.gather_fields(sp.id)
    torch.cuda.synchronize()
    assert G.check_status() & lpic.ST_HALO
    assert G.check_status() == 0                                # read and cleared
