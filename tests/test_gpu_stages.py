"""The unfused path and the species-resolved fields (the paper's callback
stages between the particle-update steps, and its Sec. 6.1 application).

* Gathering the fields into a per-particle array and pushing/depositing with
  them gives bit-identical fields, currents and particles to the fused kernel,
  and the gathered fields match the oracle's interpolation at the particles'
  half-step positions.
* A stage hook that adds a uniform B_z to the gathered fields matches the fused
  path on a grid whose B_z carries the same uniform field (to float32 rounding
  of the interpolation, which sums the shape weights).
* The species-resolved fields of a two-species laser-plasma match the oracle
  run with only that species' current as the source; with one species they
  equal the grid's own fields bit for bit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_13507_b300 import workloads as W

from pic_cases import gpu_case, oracle_case, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13507_b300 import build, lpic
    build.build()
    lpic.load()


def _unfused_step(G, t, hook=None):
    G.maxwell_half(0, t)
    G.zero_current()
    for sid in range(len(G.species)):
        f = G.gather_fields(sid)
        if hook is not None:
            hook(f)
        G.push_deposit_fields(sid, f)
    G.maxwell_half(1, t + 0.5 * G.dt)


def _by_id(sp):
    st = sp.state()
    o = np.argsort(st["id"])
    return {k: (v[..., o] if v.ndim > 1 else v[o]) for k, v in st.items()}


@pytest.mark.parametrize("case", ["thermal2d_tsc", "laser2d", "thermal3d_tsc", "thermal3d_cic"])
def test_unfused_stages_match_fused(case):
    from paper_2607_13507_b300 import lpic
    if case == "thermal2d_tsc":
        wl = W.thermal2d(n=40, ppc=6, vth=0.2, order=2, precision="fp32")
    elif case == "laser2d":
        wl = W.laser2d(nx=128, ny=32, ppc=2, precision="fp32")
    else:
        wl = W.thermal3d(n=12, ppc=3, vth=0.2, order=2 if case.endswith("tsc") else 1, precision="fp32")
    parts = W.load_all(wl)
    A = gpu_case(wl, parts, lpic.FP32_FIXED)
    B = gpu_case(wl, parts, lpic.FP32_FIXED)
    for s in range(5):
        A.step(s * wl.dt)
        _unfused_step(B, s * wl.dt)
    torch.cuda.synchronize()
    assert A.check_status() == 0 and B.check_status() == 0
    for c in range(3):
        assert torch.equal(A.E[c], B.E[c]) and torch.equal(A.B[c], B.B[c]) and torch.equal(A.J[c], B.J[c])
    for sa, sb in zip(A.species, B.species):
        a, b = _by_id(sa), _by_id(sb)
        for k in a:
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("case", ["thermal2d_tsc", "laser2d", "thermal3d_tsc"])
def test_gather_stage_matches_the_oracle_gather(case):
    """Stage 1's per-particle fields against the oracle's interpolation at
    the particles' half-step positions (x^{n+1/2}, stored cell + offsets), in
    the GPU's own fields after a few steps, to float rounding of the
    interpolation sums (1e-5 of the component's largest value)."""
    from paper_2607_13507_b300 import lpic
    if case == "thermal2d_tsc":
        wl = W.thermal2d(n=40, ppc=6, vth=0.2, order=2, precision="fp32")
    elif case == "laser2d":
        wl = W.laser2d(nx=128, ny=32, ppc=2, precision="fp32")
    else:
        wl = W.thermal3d(n=12, ppc=3, vth=0.2, order=2, precision="fp32")
    parts = W.load_all(wl)
    G = gpu_case(wl, parts, lpic.FP32_FIXED)
    steps = 30 if case == "laser2d" else 4
    for s in range(steps):
        G.step(s * wl.dt)
    t = steps * wl.dt
    G.maxwell_half(0, t)
    g = O.Grid(wl.dim, wl.n, wl.h, wl.dt, wl.order, absorb_x=wl.absorb_x)
    h = np.array(wl.h)
    rng = np.random.Generator(np.random.Philox(3))
    for sid, sp in enumerate(G.species):
        f = G.gather_fields(sid)
        torch.cuda.synchronize()
        assert G.check_status() == 0
        for c in range(3):
            g.E[c][...] = G.E[c].cpu().numpy().astype(np.float64)
            g.B[c][...] = G.B[c].cpu().numpy().astype(np.float64)
        st = sp.state()
        fg = f.cpu().numpy()
        n = st["cell"].shape[0]
        cell = st["cell"].astype(np.int64)
        coords = [cell % wl.n[0], (cell // wl.n[0]) % wl.n[1]] + ([cell // (wl.n[0] * wl.n[1])] if wl.dim == 3 else [])
        x = (np.stack(coords).astype(np.float64) + st["off"].astype(np.float64)) * h[:, None]
        pick = rng.choice(n, size=min(n, 3000), replace=False)
        scale = [max(float(torch.max(torch.abs(a)).item()), 1e-30) for a in list(G.E) + list(G.B)]
        for i in pick:
            E, B = O.gather(g, x[:, i])
            ref = np.concatenate([E, B])
            for c in range(6):
                assert abs(fg[c, i] - ref[c]) <= 1e-5 * scale[c], (sid, i, c, fg[c, i], ref[c])


def test_stage_hook_external_field():
    from paper_2607_13507_b300 import lpic
    wl = W.thermal2d(n=32, ppc=8, vth=0.05, order=2, precision="fp32")
    parts = W.load_all(wl)
    b0 = 0.7
    C = gpu_case(wl, parts, lpic.FP32_FIXED)
    C.B[2] += b0                                  # uniform B_z on the grid
    D = gpu_case(wl, parts, lpic.FP32_FIXED)

    def hook(f):
        f[5] += b0                                # the same field, added between the stages

    for s in range(3):
        C.step(s * wl.dt)
        _unfused_step(D, s * wl.dt, hook)
    torch.cuda.synchronize()
    a, b = _by_id(C.species[0]), _by_id(D.species[0])
    assert rel_l2(b["u"], a["u"]) < 1e-5
    # and the field really acted: without it the momenta differ at first order
    E = gpu_case(wl, parts, lpic.FP32_FIXED)
    for s in range(3):
        E.step(s * wl.dt)
    torch.cuda.synchronize()
    assert rel_l2(_by_id(E.species[0])["u"], a["u"]) > 1e-3


def test_stage_order_is_enforced():
    from paper_2607_13507_b300 import lpic
    wl = W.thermal2d(n=16, ppc=2, vth=0.05, order=1, precision="fp32")
    G = gpu_case(wl, W.load_all(wl), lpic.FP32_FIXED)
    f = G.gather_fields(0)
    G.push_deposit_fields(0, f)
    with pytest.raises(lpic.LpicError):
        G.push_deposit_fields(0, f)               # pushed since the gather
    G64 = gpu_case(W.thermal2d(n=16, ppc=2, order=1, precision="fp64"),
                   W.load_all(W.thermal2d(n=16, ppc=2, order=1, precision="fp64")), lpic.FP64)
    with pytest.raises(lpic.LpicError):
        G64.gather_fields(0)


def test_species_resolved_fields_match_the_oracle():
    from paper_2607_13507_b300 import lpic
    wl = W.laser2d(nx=128, ny=32, ppc=2, precision="fp64")
    parts = W.load_all(wl)
    G = gpu_case(wl, parts, lpic.FP64)
    aux = lpic.Grid(wl.dim, wl.n, wl.h, wl.dt, wl.order, lpic.FP64, absorb_x=True)
    g, sps = oracle_case(wl, parts)
    g2 = O.Grid(wl.dim, wl.n, wl.h, wl.dt, wl.order, absorb_x=True)
    sid = 0                                        # the electrons
    steps = 60
    for s in range(steps):
        t = s * wl.dt
        G.step_resolved(t, sid, aux)
        O.maxwell_half(g, 0, t)
        O.maxwell_half(g2, 0, t)
        for c in range(3):
            g.J[c][...] = 0.0
        O.push_species(g, sps[sid])
        for c in range(3):
            g2.J[c][...] = g.J[c]
        for k, sp in enumerate(sps):
            if k != sid:
                O.push_species(g, sp)
        O.maxwell_half(g, 1, t + 0.5 * wl.dt)
        O.maxwell_half(g2, 1, t + 0.5 * wl.dt)
    torch.cuda.synchronize()
    assert G.check_status() == 0
    for c in range(3):
        assert rel_l2(G.E[c].cpu().numpy(), g.E[c]) < 1e-10
        if np.linalg.norm(g2.E[c]) > 0:
            assert rel_l2(aux.E[c].cpu().numpy(), g2.E[c]) < 1e-10
        if np.linalg.norm(g2.B[c]) > 0:
            assert rel_l2(aux.B[c].cpu().numpy(), g2.B[c]) < 1e-10
    # the electrons' own field is not the total field (the laser is not in it)
    assert rel_l2(aux.E[1].cpu().numpy(), g.E[1]) > 0.1


def test_species_resolved_single_species_equals_the_total():
    from paper_2607_13507_b300 import lpic
    wl = W.thermal2d(n=32, ppc=8, vth=0.1, order=2, precision="fp32")
    G = gpu_case(wl, W.load_all(wl), lpic.FP32_FIXED)
    aux = lpic.Grid(wl.dim, wl.n, wl.h, wl.dt, wl.order, lpic.FP32_FIXED)
    for s in range(6):
        G.step_resolved(s * wl.dt, 0, aux)
    torch.cuda.synchronize()
    for c in range(3):
        assert torch.equal(aux.E[c], G.E[c]) and torch.equal(aux.B[c], G.B[c])
