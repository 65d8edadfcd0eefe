"""Cases run by the bounds test of the checked library: each exercises a
data-dependent shared-memory path of the tile kernels (the 2D deposit with
drift margins and escapes, the 3D ring of general-window moves, the 3D
laser-target's crowded and empty tiles, the form with emission, an ensemble
of mixed tilings).  run_cases(outdir) returns, per case, the status bits and
writes the final fields and current to outdir/<case>.npz; run as a script
(python checked_cases.py OUTDIR) it prints the status bits as JSON (the test
runs it with LPIC_LIBRARY pointing at the checked library)."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2607_13507_b300 import workloads as W  # noqa: E402


def _save(outdir, name, grids):
    arrays = {}
    for k, G in enumerate(grids):
        for f in ("E", "B", "J"):
            for c, t in enumerate(getattr(G, f)):
                arrays[f"g{k}_{f}{c}"] = t.cpu().numpy()
    np.savez(os.path.join(outdir, name + ".npz"), **arrays)


def run_cases(outdir):
    import torch
    from paper_2607_13507_b300 import lpic
    out = {}

    def single(name, wl, steps, **kw):
        G = lpic.grid_for(wl, lpic.FP32_FIXED, **kw)
        for p in W.load_all(wl):
            G.add_species(p)
        for s in range(steps):
            G.step(s * wl.dt)
        torch.cuda.synchronize()
        out[name] = G.check_status()
        _save(outdir, name, [G])
        G.close()

    single("laser2d_tsc_k4", W.laser2d(nx=128, ny=32, ppc=2, precision="fp32"), 24, sort_interval=4)
    single("thermal3d_tsc", W.thermal3d(n=12, ppc=3, vth=0.2, order=2, precision="fp32"), 8)
    single("laser3d_cic_k10", W.laser3d(nx=64, ny=16, nz=16, ppc=1, precision="fp32"), 30, sort_interval=10)

    # emission inside the push (fields only: photon ids follow the atomics)
    wl = W.thermal2d(n=32, ppc=1, order=2, precision="fp32")
    wl.species = []
    G = lpic.grid_for(wl, lpic.FP32_FIXED)
    G.qed_init(2e-6, 7)
    gen = W.generator(5)
    n = 256
    d = gen.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    p = W.Particles(q=-1.0, m=1.0, cell=np.stack([gen.integers(0, 32, n) for _ in range(2)]).astype(np.int32),
                    off=gen.random((2, n)).astype(np.float32),
                    u=(d * np.exp(gen.uniform(np.log(50.0), np.log(2000.0), n))).astype(np.float32),
                    w=np.ones(n, np.float32), id=np.arange(n, dtype=np.int32))
    e = G.add_species(p)
    ph = G.add_empty_species(0.0, 0.0, 4096)
    for c in range(3):
        G.B[c].fill_(300.0 if c == 2 else 0.0)
    tau = G.qed_initial_tau(n)
    G.qed_fuse(e, ph, tau)
    for s in range(4):
        G.step(s * wl.dt)
    torch.cuda.synchronize()
    out["qed_fused"] = G.check_status()
    _save(outdir, "qed_fused", [G])
    G.close()

    # ensemble with mixed tile shapes
    grids = []
    for k, (nn, tile) in enumerate((((24, 40), (8, 8)), ((40, 24), (16, 8)))):
        wl = W.thermal2d(n=nn[0], ppc=4, vth=0.1, order=1, precision="fp32", seed=500 + k)
        wl.n = nn
        G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=tile)
        G.add_species(W.load_all(wl)[0])
        grids.append(G)
    ens = lpic.Ensemble(grids)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(4):
        ens.step(side)
    torch.cuda.synchronize()
    out["ensemble_mixed"] = ens.check_status(side)
    _save(outdir, "ensemble_mixed", grids)
    ens.close()
    return out


if __name__ == "__main__":
    print(json.dumps(run_cases(sys.argv[1])))
