"""FP64 master fields on the FP32 particle path (maxwell_fp64): the Maxwell
half steps of Sec. 3.2 (Eq. 1-4) run in double with the int64 fixed-point
current converted in double, and the tile kernel rounds the fields to float
when it stages them.

* Gauss's law: div E - (rho before + rho after) / 2 stays constant over 50
  steps to 1e-12 of max |rho| (exact integer continuity of the current,
  double fields), where float fields allow only ~1e-5.
* Against the oracle: the FP32 bars after 5 steps (2D TSC, 3D CIC), and the
  200-step total-energy history of the 2D thermal plasma within 1 % of the
  oracle's.
"""
import numpy as np
import pytest

from oracle import oracle as O
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


def _grid(wl, parts, **kw):
    from paper_2607_13507_b300 import lpic
    G = lpic.grid_for(wl, lpic.FP32_FIXED, maxwell_fp64=True, **kw)
    for p in parts:
        G.add_species(p)
    assert G.E[0].dtype == torch.float64 and G.J[0].dtype == torch.int64
    return G


@pytest.mark.parametrize("dim", [2, 3])
def test_gauss_law_residual_constant_to_double_rounding(dim):
    if dim == 2:
        wl = W.thermal2d(n=32, ppc=4, vth=0.2, order=2, precision="fp32")
    else:
        wl = W.thermal3d(n=12, ppc=2, vth=0.2, order=2, precision="fp32")
    G = _grid(wl, W.load_all(wl))
    rho_prev = G.rho()
    res = []
    for s in range(50):
        G.step(s * wl.dt)
        rho = G.rho()
        res.append(G.div_e() - 0.5 * (rho + rho_prev))
        rho_prev = rho
    scale = float(rho.abs().max())
    worst = max(float((r - res[0]).abs().max()) for r in res[1:])
    assert worst < 1e-12 * scale, worst / scale
    assert G.check_status() == 0


@pytest.mark.parametrize("dim,order", [(2, 2), (3, 1)])
def test_fp64_fields_fp32_particles_against_oracle(dim, order):
    if dim == 2:
        wl = W.thermal2d(n=40, ppc=8, vth=0.05, order=order, precision="fp32")
    else:
        wl = W.thermal3d(n=12, ppc=4, vth=0.05, order=order, precision="fp32")
    parts = W.load_all(wl)
    g, sps = oracle_case(wl, parts)
    G = _grid(wl, parts)
    steps = 5
    run_oracle(g, sps, steps)
    for s in range(steps):
        G.step(s * wl.dt)
    torch.cuda.synchronize()
    assert G.check_status() == 0
    Jg = G.current()
    jtol = 1e-4 if dim == 2 else 3e-4
    for c in range(3):
        assert rel_l2(Jg[c].cpu().numpy(), g.J[c]) < jtol, ("J", c)
        assert rel_l2(G.E[c].cpu().numpy(), g.E[c]) < field_bound(jtol, steps), ("E", c)
    xg, xo, ug, uo = match_particles(G, G.species[0], sps[0], wl)
    for d in range(wl.dim):
        assert np.max(np.abs(xg[d] - xo[d])) / wl.h[d] < 1e-5
    assert rel_l2(ug, uo) < 1e-5 * steps


def test_fp64_fields_laser_edges_against_oracle():
    """Mur edges and the incoming laser in double (the edge buffers follow
    the field precision), 80 steps of the small laser-plasma, at the bound of
    the float-field test (the current's quantisation noise dominates)."""
    wl = W.laser2d(nx=128, ny=64, ppc=2, precision="fp32")
    parts = W.load_all(wl)
    g, sps = oracle_case(wl, parts)
    G = _grid(wl, parts)
    for s in range(80):
        O.step(g, sps, s * wl.dt)
        G.step(s * wl.dt)
    torch.cuda.synchronize()
    assert G.check_status() == 0
    for c in range(3):
        assert rel_l2(G.E[c].cpu().numpy(), g.E[c]) < 1e-3, ("E", c)
        assert rel_l2(G.B[c].cpu().numpy(), g.B[c]) < 1e-3, ("B", c)


def test_energy_history_200_steps_with_fp64_fields():
    wl = W.thermal2d()                       # 64 x 64, 16 per cell, 200 steps
    parts = W.load_all(wl)
    g, sps = oracle_case(wl, parts)
    G = _grid(wl, parts)
    hist_g, hist_o = [], []
    for s in range(wl.steps + 1):
        if s % 10 == 0:
            torch.cuda.synchronize()
            d = G.diagnostics()
            ek, ef, _ = O.energy(g, sps)
            hist_g.append(d.kinetic + d.field)
            hist_o.append(ek + ef)
        if s < wl.steps:
            O.step(g, sps, s * wl.dt)
            G.step(s * wl.dt)
    hist_g, hist_o = np.array(hist_g), np.array(hist_o)
    e0 = hist_o[0]
    assert np.max(np.abs(hist_g - hist_o)) < 0.01 * e0
    dg, do = hist_g - hist_g[0], hist_o - hist_o[0]
    assert np.max(np.abs(dg - do)) < 0.01 * max(np.max(np.abs(do)), 1e-3 * e0)
    assert G.check_status() == 0


def test_unsupported_combinations_are_refused():
    from paper_2607_13507_b300 import lpic
    wl = W.thermal2d(n=16, ppc=1, order=1, precision="fp32")
    G = _grid(wl, W.load_all(wl))
    with pytest.raises(lpic.LpicError):
        G.qed_init(1e-6, 1)
    with pytest.raises(lpic.LpicError):
        lpic.Ensemble([G])
