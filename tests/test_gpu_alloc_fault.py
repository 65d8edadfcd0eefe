"""Host-side fault injection (no GPU fault): the library's n-th device
allocation fails as if the device were out of memory.  Every call that
allocates -- grid creation (with Mur edges and a laser profile), species
registration, the QED tables and the fused emission's step counter, an
ensemble -- must report LPIC_ENOMEM and unwind, for every n; afterwards the
library keeps working: the same set-up succeeds once injection is off, and
its grids step bit for bit like grids built without any failure."""
import numpy as np
import pytest

from paper_2607_13507_b300 import workloads as W

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
    out = []
    for n, seed in ((24, 31), (32, 32)):
        wl = W.thermal2d(n=n, ppc=2, vth=0.05, order=1, precision="fp32", seed=seed)
        out.append(wl)
    return out


def _setup(objs):
    """Everything that allocates, in order; appends what it creates to objs."""
    from paper_2607_13507_b300 import lpic
    wl = W.laser2d(nx=64, ny=32, ppc=1, precision="fp32")      # Mur scratch and laser profile
    G = lpic.grid_for(wl, lpic.FP32_FIXED)
    objs.append(G)
    for p in W.load_all(wl):
        G.add_species(p)
    grids = []
    for k, m in enumerate(_members()):
        Gm = lpic.grid_for(m, lpic.FP32_FIXED, tile=(8, 8))
        objs.append(Gm)
        Gm.add_species(W.load_all(m)[0])
        grids.append(Gm)
    E = lpic.Ensemble(grids)
    objs.append(E)
    wq = W.thermal2d(n=16, ppc=1, order=1, precision="fp32")
    Q = lpic.grid_for(wq, lpic.FP32_FIXED)
    objs.append(Q)
    e = Q.add_species(W.load_all(wq)[0])
    ph = Q.add_empty_species(0.0, 0.0, 256)
    Q.qed_init(2e-6, 7)
    tau = Q.qed_initial_tau(256)
    Q.qed_fuse(e, ph, tau)
    return G, E, grids


def _close(objs):
    for o in reversed(objs):
        if hasattr(o, "close"):
            o.close()
    objs.clear()


def test_every_allocation_failure_unwinds_and_reports_enomem():
    from paper_2607_13507_b300 import lpic
    failed = []
    k = 1
    try:
        while True:
            objs = []
            lpic.debug_fail_alloc(k)
            try:
                _setup(objs)
                ok = True
            except lpic.LpicError as err:
                assert err.code == 2, (k, str(err))          # LPIC_ENOMEM
                ok = False
            finally:
                lpic.debug_fail_alloc(0)
                _close(objs)
            if ok:
                break
            failed.append(k)
            k += 1
            assert k < 200
    finally:
        lpic.debug_fail_alloc(0)
    # every allocation up to the last one failed in turn
    assert failed == list(range(1, k)) and len(failed) >= 40
    torch.cuda.synchronize()


def test_grids_built_after_failures_step_like_clean_ones():
    from paper_2607_13507_b300 import lpic
    # a failure in the middle of a species registration, then a clean set-up
    objs = []
    lpic.debug_fail_alloc(9)
    with pytest.raises(lpic.LpicError):
        _setup(objs)
    lpic.debug_fail_alloc(0)
    _close(objs)
    a_objs, b_objs = [], []
    Ga, Ea, ga = _setup(a_objs)
    Gb, Eb, gb = _setup(b_objs)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    for s in range(3):
        Ga.step(s * Ga.dt)
        Gb.step(s * Gb.dt)
        Ea.step(side)
        Eb.step(side)
    torch.cuda.synchronize()
    assert Ga.check_status() == 0 and Gb.check_status() == 0
    for x, y in [(Ga, Gb)] + list(zip(ga, gb)):
        for c in range(3):
            assert torch.equal(x.E[c], y.E[c]) and torch.equal(x.J[c], y.J[c])
        sa, sb = x.species[0].state(), y.species[0].state()
        oa, ob = np.argsort(sa["id"]), np.argsort(sb["id"])
        assert np.array_equal(sa["u"][:, oa], sb["u"][:, ob])
    _close(a_objs)
    _close(b_objs)
