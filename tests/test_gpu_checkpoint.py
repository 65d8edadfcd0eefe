"""Checkpoint and resume: all state is caller-owned tensors (fields, integer
current, particle buffers) plus each species' weight bound (which fixes the
fixed-point shift) and next created id.  A run saved to a file half-way and
restored into a freshly created grid ends where the uninterrupted run ends:
bit for bit on the FP32 path (its integer deposit does not depend on the
particle order, and the restored grid sorts at a different step), to double
rounding on the FP64 path (its double atomics add in a varying order)."""
import numpy as np
import pytest

from paper_2607_13507_b300 import workloads as W

from pic_cases import gpu_case, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13507_b300 import build, lpic
    build.build()
    lpic.load()


def _by_id(sp):
    st = sp.state()
    keep = st["cell"] >= 0 if "cell" in st else np.ones(st["id"].shape[0], bool)
    o = np.argsort(st["id"][keep])
    return {k: (v[..., keep][..., o] if v.ndim > 1 else v[keep][o]) for k, v in st.items()}


@pytest.mark.parametrize("case", ["laser2d_fp32", "thermal3d_fp32", "thermal2d_fp64"])
def test_resume_from_file_continues_the_run(case, tmp_path):
    from paper_2607_13507_b300 import lpic
    if case == "laser2d_fp32":
        wl, prec, steps = W.laser2d(nx=128, ny=32, ppc=2, precision="fp32"), lpic.FP32_FIXED, 40
    elif case == "thermal3d_fp32":
        wl, prec, steps = W.thermal3d(n=12, ppc=3, vth=0.2, order=1, precision="fp32"), lpic.FP32_FIXED, 12
    else:
        wl, prec, steps = W.thermal2d(n=32, ppc=4, vth=0.05, order=2, precision="fp64"), lpic.FP64, 12
    parts = W.load_all(wl)
    A = gpu_case(wl, parts, prec)
    B = gpu_case(wl, parts, prec)
    half = steps // 2
    for s in range(steps):
        A.step(s * wl.dt)
    for s in range(half):
        B.step(s * wl.dt)
    path = tmp_path / "state.npz"
    lpic.save_checkpoint(B, path)
    B.close()
    C = lpic.grid_for(wl, prec)
    lpic.load_checkpoint(C, path)
    for s in range(half, steps):
        C.step(s * wl.dt)
    torch.cuda.synchronize()
    assert A.check_status() == 0 and C.check_status() == 0
    exact = prec == lpic.FP32_FIXED
    for name in ("E", "B", "J"):
        for a, c in zip(getattr(A, name), getattr(C, name)):
            if exact:
                assert torch.equal(a, c), name
            else:
                assert rel_l2(c.cpu().numpy(), a.cpu().numpy()) < 1e-12, name
    for sa, sc in zip(A.species, C.species):
        a, c = _by_id(sa), _by_id(sc)
        assert np.array_equal(a["id"], c["id"])
        for k in a:
            if exact:
                assert np.array_equal(a[k], c[k]), k
            else:
                assert rel_l2(c[k], a[k]) < 1e-12, k


def test_restore_refuses_a_grid_with_species_or_another_shape(tmp_path):
    from paper_2607_13507_b300 import lpic
    wl = W.thermal2d(n=16, ppc=2, order=1, precision="fp32")
    parts = W.load_all(wl)
    A = gpu_case(wl, parts, lpic.FP32_FIXED)
    A.step(0.0)
    ck = A.checkpoint()
    with pytest.raises(ValueError):
        A.restore(ck)                         # already holds species
    other = lpic.grid_for(W.thermal2d(n=24, ppc=2, order=1, precision="fp32"), lpic.FP32_FIXED)
    with pytest.raises(ValueError):
        other.restore(ck)
