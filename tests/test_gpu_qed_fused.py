"""Nonlinear Compton emission inside the fused particle kernel (Algorithm 1:
QED events between the field interpolation and the momentum push) against
the oracle's particle loop with the same placement, and the step plumbing
around it (device counter word, photon push in the same step, graph
replays, refusals).  The event bars are those of the separate emission pass
(the same float table lookups): decisions equal except where the depth left
is within the rate tolerance of zero, depths decremented alike (5e-4 of the
decrement) and restarted alike (2e-6), photon momenta 1e-3 and directions
1e-5; the push and deposit at the FP32 plasma bars (positions 1e-5 cell,
momenta 1e-5 relative plus the recoil's 1e-3 of k, J 1e-4 relative L2)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_13507_b300 import workloads as W

from pic_cases import field_bound, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEED = 0x5EED0F0B


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13507_b300 import build, lpic
    build.build()
    lpic.load()


def _grid(dim, order, eps_ref=2e-6, n=None, sort_interval=0):
    from paper_2607_13507_b300 import lpic
    if dim == 2:
        wl = W.thermal2d(n=n or 32, ppc=1, order=order, precision="fp32")
    else:
        wl = W.thermal3d(n=n or 8, ppc=1, order=order, precision="fp32")
    wl.species = []
    G = lpic.grid_for(wl, lpic.FP32_FIXED, sort_interval=sort_interval)
    G.qed_init(eps_ref, SEED)
    g = O.Grid(dim, wl.n, wl.h, wl.dt, order)
    return wl, G, g


def _fields(G, g, wl, F0):
    """Smooth fields varying along every axis, the same float values on both sides."""
    nz, ny, fx = G.field_shape
    x = np.arange(fx)[None, None, :] * wl.h[0]
    y = np.arange(ny)[None, :, None] * wl.h[1]
    z = (np.arange(nz)[:, None, None] * wl.h[2]) if wl.dim == 3 else np.zeros((1, 1, 1))
    L = [wl.n[d] * wl.h[d] for d in range(wl.dim)] + ([1.0] if wl.dim == 2 else [])
    kx, ky, kz = (2 * np.pi / l for l in L)
    vals = [0.1 * F0 * np.sin(ky * y + kz * z), F0 * (1 + 0.3 * np.sin(kx * x)) * (1 + 0.1 * np.cos(kz * z)),
            0.2 * F0 * np.cos(kx * x + ky * y), 0.05 * F0 * np.cos(ky * y), 0.1 * F0 * np.sin(kx * x + kz * z),
            F0 * (1 + 0.2 * np.cos(ky * y)) * (1 + 0.1 * np.sin(kz * z))]
    for c in range(6):
        v32 = (vals[c] * np.ones((nz, ny, fx))).astype(np.float32)
        (G.E + G.B)[c].copy_(torch.from_numpy(v32).to(G.device))
        (g.E + g.B)[c][...] = v32.astype(np.float64)


def _beam(wl, n, seed, umin, umax, q=-1.0):
    gen = W.generator(seed)
    cell = np.stack([gen.integers(0, wl.n[d], n) for d in range(wl.dim)]).astype(np.int32)
    off = gen.random((wl.dim, n)).astype(np.float32)
    d = gen.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    mag = np.exp(gen.uniform(np.log(umin), np.log(umax), n))
    return W.Particles(q=q, m=1.0, cell=cell, off=off, u=(d * mag).astype(np.float32),
                       w=np.ones(n, np.float32), id=np.arange(n, dtype=np.int32))


def _by_id(st, key):
    o = np.argsort(st["id"])
    v = st[key]
    return v[:, o] if v.ndim == 2 else v[o]


def _owners(st_e0, st_ph, new):
    """Each new device photon's emitter: the photon starts at the emitter's
    stored position before the push (the same cell and offsets)."""
    dim = st_e0["off"].shape[0]
    key = {(int(c),) + tuple(float(st_e0["off"][d][k]) for d in range(dim)): int(i)
           for k, (c, i) in enumerate(zip(st_e0["cell"], st_e0["id"]))}
    idx = np.nonzero(new)[0]
    return np.array([key[(int(st_ph["cell"][k]),) + tuple(float(st_ph["off"][d][k]) for d in range(dim))]
                     for k in idx], dtype=np.int64), idx


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_fused_emission_pushes_match_oracle(dim, order):
    # chi ~ 0.1 .. 10 on both grids (3D: weaker fields with a larger eps_ref,
    # so that one step turns a momentum by a moderate angle)
    eps = 2e-6 if dim == 2 else 1e-5
    wl, G, g = _grid(dim, order, eps)
    n = 160 if dim == 2 else 96
    p = _beam(wl, n, seed=31 + 10 * dim + order, umin=50.0 if dim == 2 else 20.0,
              umax=2000.0 if dim == 2 else 400.0)
    e = G.add_species(p)                       # stored at x + (dt/2) v
    ph = G.add_empty_species(0.0, 0.0, 8 * n)
    h = np.array(wl.h)[:, None]
    so = O.Species(p.q, p.m, (p.cell + p.off) * h, p.u.astype(np.float64), p.w.astype(np.float64))
    _fields(G, g, wl, 800.0 if dim == 2 else 4e3)
    tau_g = G.qed_initial_tau(n)
    tau_o = O.qed_initial_tau(np.arange(n), SEED)
    G.qed_fuse(e, ph, tau_g, first_step=0)
    ok = np.ones(n, bool)
    xbud = np.zeros(n)
    events = 0
    for step in range(3):
        G.sort(e.id)
        st0 = e.state()
        u0_g = _by_id(st0, "u").astype(np.float64)
        u0_o = so.u.copy()
        ph_before = set(ph.state()["id"].tolist())
        t0_o = tau_o.copy()
        G.qed_set_step(step)
        G.zero_current()
        G.gather_push_deposit(e.id)
        for c in range(3):
            g.J[c][...] = 0.0
        phot_o, own_o = O.push_species_qed(g, so, eps, SEED, step, tau_o)
        torch.cuda.synchronize()
        assert G.check_status() == 0
        st1 = e.state()
        stp = ph.state()
        t1_g = tau_g.cpu().numpy().astype(np.float64)
        new = np.array([i not in ph_before for i in stp["id"]], dtype=bool)
        own_g, idx = _owners(st0, stp, new)
        assert len(set(own_g.tolist())) == len(own_g)
        em_g = np.zeros(n, bool)
        em_g[own_g] = True
        em_o = np.zeros(n, bool)
        em_o[own_o] = True
        mis = ok & (em_g != em_o)
        for i in np.nonzero(mis)[0]:
            rest = t1_g[i] if em_o[i] else tau_o[i]
            assert rest < 1e-3 * max(t0_o[i], 1.0) + 1e-4, (i, rest)
        assert mis.sum() <= max(2, n // 100)
        both, none = ok & em_g & em_o, ok & ~em_g & ~em_o
        events += int(both.sum())
        dec_o = t0_o[none] - tau_o[none]
        assert np.all(np.abs(t1_g[none] - tau_o[none]) <= 5e-4 * dec_o + 2e-6 * t0_o[none] + 1e-5)
        np.testing.assert_allclose(t1_g[both], tau_o[both], rtol=2e-6)
        # photons: k u^n/|u^n| with the emitter's weight
        kv_g = np.zeros((3, n))
        kv_g[:, own_g] = stp["u"][:, idx].astype(np.float64)
        kv_o = np.zeros((3, n))
        kv_o[:, own_o] = phot_o.u
        k_g, k_o = np.linalg.norm(kv_g, axis=0), np.linalg.norm(kv_o, axis=0)
        assert np.all(np.abs(k_g[both] - k_o[both]) <= 1e-3 * k_o[both])
        dg = kv_g[:, both] / k_g[both]
        # the emitters' momenta already differ by what earlier steps left
        # (|du| turns the direction by at most 2 |du| / |u|)
        before = np.linalg.norm(u0_g - u0_o, axis=0)
        turn = 2.0 * before / np.linalg.norm(u0_o, axis=0)
        assert np.all(np.linalg.norm(dg - kv_o[:, both] / k_o[both], axis=0) < 1e-5 + turn[both])
        # the photon leaves along the emitter's momentum before the push
        assert np.all(np.linalg.norm(dg - u0_g[:, both] / np.linalg.norm(u0_g[:, both], axis=0), axis=0) < 2e-6)
        assert np.all(stp["w"][idx] == 1.0)
        # the push of the recoiled momentum
        u1_g = _by_id(st1, "u").astype(np.float64)
        err = np.linalg.norm(u1_g - so.u, axis=0)
        bound = before + 1e-3 * k_o + 1e-5 * np.linalg.norm(so.u, axis=0) + 1e-5
        assert np.all(err[ok & ~mis] <= bound[ok & ~mis]), np.max((err - bound)[ok & ~mis])
        # positions at the integer time (a velocity off by |du| at most moves
        # the particle |du| dt further) and the current
        x1 = e.positions_at_step()[:, np.argsort(st1["id"])]
        xbud += err * wl.dt
        for d in range(dim):
            L = wl.n[d] * wl.h[d]
            diff = np.remainder(x1[d] - so.x[d] + 0.5 * L, L) - 0.5 * L
            sel = ok & ~mis
            assert np.all(np.abs(diff[sel]) <= 1e-5 * (step + 1) * wl.h[d] + xbud[sel]), d
        if mis.sum() == 0 and ok.all():
            Jg = G.current()
            for c in range(3):
                if np.linalg.norm(g.J[c]) > 0:
                    assert rel_l2(Jg[c].cpu().numpy(), g.J[c]) < 1e-4, ("J", c)
        ok &= ~mis
    assert events > n // 6


def _plasma_case(order=2, n_cells=32, seed=5, sort_interval=0):
    """An electron-positron beam mix in strong fields: photons pile up in a
    photon species added after the leptons."""
    from paper_2607_13507_b300 import lpic
    wl, G, g = _grid(2, order, 2e-6, n=n_cells, sort_interval=sort_interval)
    el = _beam(wl, 200, seed, 50.0, 1500.0, q=-1.0)
    po = _beam(wl, 200, seed + 1, 50.0, 1500.0, q=1.0)
    po = W.Particles(q=1.0, m=1.0, cell=po.cell, off=po.off, u=po.u, w=po.w,
                     id=(np.arange(200) + 200).astype(np.int32))
    e = G.add_species(el)
    p = G.add_species(po)
    ph = G.add_empty_species(0.0, 0.0, 8192)
    _fields(G, g, wl, 600.0)
    tau = G.qed_initial_tau(400)
    G.qed_fuse(e, ph, tau, first_step=0)
    G.qed_fuse(p, ph, tau, first_step=0)
    return wl, G, g, (e, p, ph), tau, (el, po)


@pytest.mark.parametrize("sort_interval", [1, 4])
def test_fused_emission_steps_match_oracle(sort_interval):
    """Four full steps (Maxwell halves, both leptons emitting into one photon
    species, photons pushed in the same step) against the oracle doing the
    same with its particle loop and photon push; with a sort every 4 steps
    the particles that drift past their tile's margin take the emission in
    the escape kernel."""
    wl, G, g, (e, p, ph), tau_g, (el, po) = _plasma_case(sort_interval=sort_interval)
    h = np.array(wl.h)[:, None]
    so = [O.Species(q.q, q.m, (q.cell + q.off) * h, q.u.astype(np.float64), q.w.astype(np.float64))
          for q in (el, po)]
    tau_o = [O.qed_initial_tau(np.arange(200), SEED), O.qed_initial_tau(np.arange(200) + 200, SEED)]
    phot = O.Species(0.0, 0.0, np.zeros((2, 0)), np.zeros((3, 0)), np.zeros(0))
    # the oracle draws counter (index, step, 0, 0): its positron ids are
    # offset by 200, as on the device, through a padded depth array
    steps = 4
    for s in range(steps):
        t = s * wl.dt
        O.maxwell_half(g, 0, t)
        for c in range(3):
            g.J[c][...] = 0.0
        new = []
        for k, sp in enumerate(so):
            if k == 0:
                pn, _ = O.push_species_qed(g, sp, 2e-6, SEED, s, tau_o[0])
            else:
                # positrons carry ids 200.. : run them as the tail of a padded species
                pad = O.Species(sp.q, sp.m, np.concatenate([np.zeros((2, 200)), sp.x[:2]], 1),
                                np.concatenate([np.zeros((3, 200)), sp.u], 1),
                                np.concatenate([np.zeros(200), sp.w]),
                                alive=np.concatenate([np.zeros(200, np.int32), sp.alive]))
                tpad = np.concatenate([np.zeros(200), tau_o[1]])
                pn, _ = O.push_species_qed(g, pad, 2e-6, SEED, s, tpad)
                sp.x[:2], sp.u[...] = pad.x[:2, 200:], pad.u[:, 200:]
                tau_o[1][...] = tpad[200:]
            new.append(pn)
        O.push_species(g, phot)
        xs = [phot.x[:2]] + [q.x[:2] for q in new]
        us = [phot.u] + [q.u for q in new]
        ws = [phot.w] + [q.w for q in new]
        phot = O.Species(0.0, 0.0, np.concatenate(xs, 1), np.concatenate(us, 1), np.concatenate(ws))
        O.maxwell_half(g, 1, t + 0.5 * wl.dt)
        G.step(t)
    torch.cuda.synchronize()
    assert G.check_status() == 0
    Jg = G.current()
    for c in range(3):
        assert rel_l2(Jg[c].cpu().numpy(), g.J[c]) < 1e-4, ("J", c)
        assert rel_l2(G.E[c].cpu().numpy(), g.E[c]) < field_bound(1e-4, steps), ("E", c)
        assert rel_l2(G.B[c].cpu().numpy(), g.B[c]) < field_bound(1e-4, steps), ("B", c)
    # photons: as many (up to decisions at the rate margin), each matched by
    # direction, with its momentum and its position at the integer time
    stp = ph.state()
    xg = ph.positions_at_step()
    ng, no = stp["id"].shape[0], phot.x.shape[1]
    assert no > 100
    assert abs(ng - no) <= max(2, no // 100)
    dg = stp["u"].astype(np.float64)
    dg = dg / np.linalg.norm(dg, axis=0)
    do = phot.u / np.linalg.norm(phot.u, axis=0)
    matched = 0
    for j in range(no):
        k = int(np.argmax(do[:, j] @ dg))
        if np.linalg.norm(dg[:, k] - do[:, j]) > 1e-4:
            continue                                   # a photon the device did not emit
        matched += 1
        assert abs(np.linalg.norm(stp["u"][:, k]) / np.linalg.norm(phot.u[:, j]) - 1.0) < 1e-3
        for d in range(2):
            L = wl.n[d] * wl.h[d]
            diff = np.remainder(xg[d, k] - phot.x[d, j] + 0.5 * L, L) - 0.5 * L
            assert abs(diff) / wl.h[d] < 1e-4
    assert matched >= no - max(2, no // 100)


def test_fused_emission_graph_replays_match_eager_steps():
    wl, Ga, _, (ea, pa, pha), tau_a, _ = _plasma_case(seed=9)
    wl, Gb, _, (eb, pb, phb), tau_b, _ = _plasma_case(seed=9)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    for s in range(5):
        Ga.step(s * wl.dt)
    Gb.set_clock(0.0, side)
    Gb.graph_steps(2, side)
    Gb.graph_steps(3, side)
    torch.cuda.synchronize()
    assert Ga.check_status() == 0 and Gb.check_status() == 0
    for c in range(3):
        assert torch.equal(Ga.E[c], Gb.E[c]) and torch.equal(Ga.B[c], Gb.B[c]) and torch.equal(Ga.J[c], Gb.J[c])
    assert torch.equal(tau_a, tau_b)
    for a, b in ((ea, eb), (pa, pb)):
        sa, sb = a.state(), b.state()
        oa, ob = np.argsort(sa["id"]), np.argsort(sb["id"])
        assert np.array_equal(sa["id"][oa], sb["id"][ob])
        assert np.array_equal(sa["u"][:, oa], sb["u"][:, ob])
        assert np.array_equal(sa["cell"][oa], sb["cell"][ob])
    # photon ids follow the order of the atomic slots: compare the sets of momenta
    ua = np.sort(pha.state()["u"][0])
    ub = np.sort(phb.state()["u"][0])
    assert np.array_equal(ua, ub)


def test_fused_photon_overflow_leaves_emitters_untouched():
    """More emissions than photon slots: the status is raised, as many
    photons as slots are created, and an emitter left without a photon is
    pushed without recoil and keeps its spent depth."""
    from paper_2607_13507_b300 import lpic
    wl, G, g = _grid(2, 1)
    n = 1024
    p = _beam(wl, n, seed=5, umin=50.0, umax=2000.0)
    e = G.add_species(p)
    ph = G.add_empty_species(0.0, 0.0, 64)
    _fields(G, g, wl, 200.0)
    tau = torch.zeros(n, dtype=torch.float32, device=G.device)    # every particle emits
    G.qed_fuse(e, ph, tau, first_step=0)
    # the same push without emission, on a second grid
    G2 = lpic.grid_for(wl, lpic.FP32_FIXED)
    e2 = G2.add_species(p)
    for c in range(3):
        G2.E[c].copy_(G.E[c])
        G2.B[c].copy_(G.B[c])
    for GG, sp in ((G, e), (G2, e2)):
        GG.sort(sp.id)
        GG.zero_current()
        GG.gather_push_deposit(sp.id)
    bits = G.check_status()
    assert bits & lpic.ST_OVERFLOW
    assert G2.check_status() == 0
    assert ph.query()[1] == 64
    t = tau.cpu().numpy()
    s1, s2 = e.state(), e2.state()
    emitted = t[np.sort(s1["id"])] > 0
    assert emitted.sum() == 64
    u1, u2 = _by_id(s1, "u"), _by_id(s2, "u")
    assert np.array_equal(u1[:, ~emitted], u2[:, ~emitted])
    assert np.all(t[np.sort(s1["id"])][~emitted] <= 0)
    assert not np.array_equal(u1[:, emitted], u2[:, emitted])


def test_fused_emission_refusals():
    from paper_2607_13507_b300 import lpic
    wl, G, g = _grid(2, 1)
    ph = G.add_empty_species(0.0, 0.0, 64)
    e = G.add_species(_beam(wl, 64, seed=3, umin=10.0, umax=20.0))
    tau = G.qed_initial_tau(64)
    with pytest.raises(lpic.LpicError):
        G.qed_fuse(e, ph, tau)                 # photon species listed before the emitter
    ph2 = G.add_empty_species(0.0, 0.0, 64)
    with pytest.raises(lpic.LpicError):
        G.qed_fuse(ph, ph2, tau)               # massless emitter
    G.qed_fuse(e, ph2, tau)
    with pytest.raises(lpic.LpicError):
        G.gather_fields(e.id)                  # no unfused stages with emission
    with pytest.raises(lpic.LpicError):
        lpic.Ensemble([G])
    G.qed_fuse(e, None, None)                  # off again: the stages run
    G.gather_fields(e.id)
    torch.cuda.synchronize()
    assert G.check_status() == 0
