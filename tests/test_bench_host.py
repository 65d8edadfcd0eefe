"""Host-side pieces of bench.py that need no GPU: the threaded oracle step
used for the CPU baseline gives the plain oracle step's fields (the private
currents are summed in another order, so to rounding)."""
import numpy as np
import pytest

import bench
from oracle import oracle as O
from paper_2607_13507_b300 import workloads as W


@pytest.mark.parametrize("name,threads", [("thermal3d", 4), ("laser2d", 3)])
def test_threaded_oracle_step_matches_plain_step(name, threads):
    if name == "thermal3d":
        wl = W.thermal3d(n=10, ppc=3, precision="fp64")
    else:
        wl = W.laser2d(nx=64, ny=16, ppc=4, precision="fp64")
    parts = W.load_all(wl)
    h = np.array(wl.h)[:, None]
    g1 = O.Grid(wl.dim, wl.n, wl.h, wl.dt, wl.order, absorb_x=wl.absorb_x)
    g2 = O.Grid(wl.dim, wl.n, wl.h, wl.dt, wl.order, absorb_x=wl.absorb_x)
    s1 = [O.Species(p.q, p.m, (p.cell + p.off) * h, p.u, p.w) for p in parts]
    s2 = [O.Species(p.q, p.m, (p.cell + p.off) * h, p.u, p.w) for p in parts]
    step = bench._ThreadedOracleStep(O, g2, s2, threads)
    assert step.alive() == sum(int(s.alive.sum()) for s in s1)
    for k in range(3):
        O.step(g1, s1, k * wl.dt)
        step(k * wl.dt)
    for c in range(3):
        for a, b in ((g1.E[c], g2.E[c]), (g1.B[c], g2.B[c]), (g1.J[c], g2.J[c])):
            scale = max(np.abs(a).max(), 1e-300)
            assert np.abs(a - b).max() <= 1e-13 * scale
    # the slices carry the same particles as the plain species
    u2 = np.concatenate([part.u for _, part in step.jobs], axis=1)
    u1 = np.concatenate([s.u for s in s1], axis=1)
    assert np.abs(np.sort(u1.ravel()) - np.sort(u2.ravel())).max() < 1e-13
