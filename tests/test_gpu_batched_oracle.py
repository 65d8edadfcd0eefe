"""The batched paths against the FP64 oracle, element by element: members of
an ensemble (uneven periodic 2D plasmas stepped together: batched field and
sort kernels, one persistent particle kernel over a device work queue),
eagerly and from replayed CUDA graphs, and a single grid stepped from
replayed graphs, each compared with the oracle stepping the same member
alone, at the FP32 bars of the single-grid parity tests (J <= 1e-4, E and B
<= 1e-4 per step relative L2; particles matched by id, positions <= 1e-5
cell, momenta <= 1e-5 per step)."""
import numpy as np
import pytest

from paper_2607_13507_b300 import workloads as W

from pic_cases import field_bound, match_particles, oracle_case, rel_l2, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13507_b300 import build, lpic
    build.build()
    lpic.load()


def _members():
    # uneven sides, particles per cell and temperatures, like the ensemble
    # workload at small sizes
    spec = [((40, 48), 4, 0.05, 901), ((56, 32), 8, 0.08, 902), ((32, 64), 12, 0.03, 903)]
    out = []
    for n, ppc, vth, seed in spec:
        wl = W.thermal2d(n=n[0], ppc=ppc, vth=vth, order=1, precision="fp32", seed=seed)
        wl.n = n
        out.append(wl)
    return out


def _compare(G, g, sps, wl, steps):
    Jg = G.current()
    jtol = 1e-4
    for c in range(3):
        assert rel_l2(Jg[c].cpu().numpy(), g.J[c]) < jtol, ("J", c)
        assert rel_l2(G.E[c].cpu().numpy(), g.E[c]) < field_bound(jtol, steps), ("E", c)
        if np.linalg.norm(g.B[c]) > 0:
            assert rel_l2(G.B[c].cpu().numpy(), g.B[c]) < field_bound(jtol, steps), ("B", c)
    xg, xo, ug, uo = match_particles(G, G.species[0], sps[0], wl)
    for d in range(wl.dim):
        assert np.max(np.abs(xg[d] - xo[d])) / wl.h[d] < 1e-5
    assert rel_l2(ug, uo) < 1e-5 * steps


@pytest.mark.parametrize("mode", ["eager", "graph"])
def test_ensemble_members_match_oracle(mode):
    from paper_2607_13507_b300 import lpic
    wls = _members()
    grids, orc = [], []
    # members keep their own tile shapes and particles per block
    launch = [((8, 8), 2048), ((16, 8), 4096), ((16, 16), 8192)]
    for wl, (tile, P) in zip(wls, launch):
        parts = W.load_all(wl)
        G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=tile, block_particles=P)
        G.add_species(parts[0])
        grids.append(G)
        orc.append(oracle_case(wl, parts))
    ens = lpic.Ensemble(grids)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    steps = 5
    if mode == "eager":
        for _ in range(steps):
            ens.step(side)
    else:
        ens.graph_steps(2, side)
        ens.graph_steps(3, side)
    torch.cuda.synchronize()
    assert ens.check_status(side) == 0
    ens.close()
    for G, wl, (g, sps) in zip(grids, wls, orc):
        run_oracle(g, sps, steps)
        _compare(G, g, sps, wl, steps)


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 1)])
def test_graph_replay_matches_oracle(dim, order):
    from paper_2607_13507_b300 import lpic
    if dim == 2:
        wl = W.thermal2d(n=40, ppc=8, vth=0.05, order=order, precision="fp32")
    else:
        wl = W.thermal3d(n=12, ppc=4, vth=0.05, order=order, precision="fp32")
    parts = W.load_all(wl)
    G = lpic.grid_for(wl, lpic.FP32_FIXED)
    G.add_species(parts[0])
    g, sps = oracle_case(wl, parts)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    steps = 5
    G.set_clock(0.0, side)
    G.graph_steps(2, side)
    G.graph_steps(3, side)
    torch.cuda.synchronize()
    assert G.check_status() == 0
    run_oracle(g, sps, steps)
    _compare(G, g, sps, wl, steps)
