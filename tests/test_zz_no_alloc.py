"""The allocation-free tile sort (lpic_sort_tiles_static) gives the same
result as the grid's own sort (lpic_sort_particles).

It exists for callers that cannot allocate device memory (a host framework
that owns all device memory through its own pool, code running while a graph
is being captured in global mode, a real-time loop that cannot take the
synchronisation of cudaMalloc).  This file is collected last so that a run
that stops at its first failure has already run every other test; it also
passes on its own in a fresh process.

The order of particles inside a tile is not specified, so the comparison is:
the same alive count, the same tile boundaries, the same set of ids in every
tile, and bit-identical per-particle state for every id.
"""
import ctypes

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


def _arrays(buf_u8, cap, dim, n):
    """Views (cell, off, u, w, id) of the first n entries of an FP32 buffer."""
    a = 4 * cap
    seg = lambda k, dt: buf_u8[k * a: (k + 1) * a].view(dt)[:n].cpu().numpy()
    return dict(cell=seg(0, torch.int32),
                off=np.stack([seg(1 + d, torch.float32) for d in range(dim)]),
                u=np.stack([seg(1 + dim + c, torch.float32) for c in range(3)]),
                w=seg(4 + dim, torch.float32), id=seg(5 + dim, torch.int32))


def _tile_key(cell, nx, ny, T, dim):
    x, r = cell % nx, cell // nx
    y, z = r % ny, r // ny
    ntx = (nx + T[0] - 1) // T[0]
    nty = (ny + T[1] - 1) // T[1]
    key = (y // T[1]) * ntx + x // T[0]
    if dim == 3:
        key = key + (z // T[2]) * ntx * nty
    return key


def _static_sort(G, sp, dst_u8, tile):
    from paper_2607_13507_b300 import lpic
    L = lpic.load()
    cur, n = sp.query()
    src_ptr = sp.ptr(cur)
    cnt_in = torch.tensor([n], dtype=torch.int32, device="cuda")
    cnt_out = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    nt = 1
    for d in range(G.dim):
        nt *= (G.n[d] + tile[d] - 1) // tile[d]
    starts = torch.full((nt + 1,), -7, dtype=torch.int32, device="cuda")
    t3 = (ctypes.c_int * 3)(*(list(tile) + [1] * (3 - len(tile))))
    rc = L.lpic_sort_tiles_static(G.dim, G.n[0], G.n[1], G.n[2], t3, src_ptr, dst_u8.data_ptr(),
                                  sp.cap, cnt_in.data_ptr(), cnt_out.data_ptr(), starts.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == 0, L.lpic_last_error()
    torch.cuda.synchronize()
    return int(cnt_out.item()), starts.cpu().numpy()


def _compare(G, sp, tile, got, n_got, starts):
    """Static-sort output `got` against the grid sort of the same input."""
    G.sort(sp.id)
    ref = sp.state()
    n_ref = ref["id"].shape[0]
    assert n_got == n_ref
    assert starts[-1] == n_ref
    key_ref = _tile_key(ref["cell"], G.n[0], G.n[1], tile, G.dim)
    key_got = _tile_key(got["cell"], G.n[0], G.n[1], tile, G.dim)
    assert np.all(np.diff(key_got) >= 0)
    bounds = np.searchsorted(key_ref, np.arange(len(starts) - 1), side="left")
    assert np.array_equal(bounds, starts[:-1])
    for t in range(len(starts) - 1):
        a = np.sort(got["id"][starts[t]:starts[t + 1]])
        b = np.sort(ref["id"][starts[t]:starts[t + 1]])
        assert np.array_equal(a, b)
    og, orf = np.argsort(got["id"]), np.argsort(ref["id"])
    for k in ("cell", "w"):
        assert np.array_equal(got[k][og], ref[k][orf])
    for k in ("off", "u"):
        assert np.array_equal(got[k][:, og], ref[k][:, orf])


@pytest.mark.parametrize("dim", [2, 3])
def test_static_sort_matches_grid_sort_on_two_calls(dim):
    from paper_2607_13507_b300 import lpic
    if dim == 2:
        wl = W.thermal2d(n=48, ppc=5, vth=0.2, order=2, precision="fp32")
        tile = (16, 8)
    else:
        wl = W.thermal3d(n=12, ppc=3, vth=0.2, order=1, precision="fp32")
        tile = (4, 8, 6)
    G = lpic.grid_for(wl, lpic.FP32_FIXED, tile=tile)
    sp = G.add_species(W.load_all(wl)[0])
    dst = torch.zeros(lpic.species_bytes(G.dim, lpic.FP32_FIXED, sp.cap) + 512, dtype=torch.uint8,
                      device="cuda")
    off = (-dst.data_ptr()) % 256
    dst_u8 = dst[off:]
    for call in range(2):
        # mark one particle removed so the compaction is exercised
        cur, n = sp.query()
        sp._views(cur)["cell"][3 + call] = -1
        n_got, starts = _static_sort(G, sp, dst_u8, tile)
        got = _arrays(dst_u8, sp.cap, G.dim, n_got)
        _compare(G, sp, tile, got, n_got, starts)
        # move the particles so the second call sorts a different state
        G.zero_current()
        G.gather_push_deposit(sp.id)
        torch.cuda.synchronize()
    assert G.check_status() == 0


def test_static_sort_rejects_too_many_tiles():
    from paper_2607_13507_b300 import lpic
    L = lpic.load()
    t3 = (ctypes.c_int * 3)(1, 1, 1)
    # real, aligned device buffers, so that no order of the host checks can
    # hand the kernels an invalid address
    nbytes = lpic.species_bytes(2, lpic.FP32_FIXED, 64)
    src = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    dst = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    s_ptr = src.data_ptr() + (-src.data_ptr()) % 256
    d_ptr = dst.data_ptr() + (-dst.data_ptr()) % 256
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    starts = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = L.lpic_sort_tiles_static(2, 512, 512, 1, t3, s_ptr, d_ptr, 64, cnt.data_ptr(),
                                  cnt.data_ptr() + 4, starts.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == 1
    assert b"LPIC_NOALLOC_MAX_TILES" in L.lpic_last_error()
    torch.cuda.synchronize()


def test_static_sort_clamps_count_and_drops_cells_off_the_grid():
    """A count above the capacity is taken as the capacity and a cell at or
    beyond nx ny is dropped like a removed particle: nothing outside dst, the
    counts and the starts is written."""
    from paper_2607_13507_b300 import lpic
    L = lpic.load()
    nx, ny, tile, cap = 16, 8, (8, 4), 64
    nbytes = lpic.species_bytes(2, lpic.FP32_FIXED, cap)
    src = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    guard = 4096
    dst = torch.full((nbytes + 256 + guard,), 0xA5, dtype=torch.uint8, device="cuda")
    s_off = (-src.data_ptr()) % 256
    d_off = (-dst.data_ptr()) % 256
    rng = np.random.default_rng(5)
    cell = rng.integers(0, nx * ny, cap).astype(np.int32)
    cell[3] = nx * ny            # just off the grid
    cell[9] = 1 << 30            # far off the grid
    cell[20] = -1                # removed
    ids = np.arange(cap, dtype=np.int32)
    a = 4 * cap
    body = src[s_off:s_off + nbytes]
    body[0:a].view(torch.int32).copy_(torch.from_numpy(cell))
    for k in range(1, 7):
        body[k * a:(k + 1) * a].view(torch.float32).copy_(torch.from_numpy(rng.random(cap).astype(np.float32)))
    body[7 * a:8 * a].view(torch.int32).copy_(torch.from_numpy(ids))
    cnt_in = torch.tensor([10 * cap], dtype=torch.int32, device="cuda")
    cnt_out = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    nt = (nx // tile[0]) * (ny // tile[1])
    starts = torch.full((nt + 1 + 64,), -7, dtype=torch.int32, device="cuda")
    t3 = (ctypes.c_int * 3)(tile[0], tile[1], 1)
    for _ in range(2):
        rc = L.lpic_sort_tiles_static(2, nx, ny, 1, t3, src.data_ptr() + s_off, dst.data_ptr() + d_off,
                                      cap, cnt_in.data_ptr(), cnt_out.data_ptr(), starts.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
        assert rc == 0, L.lpic_last_error()
        torch.cuda.synchronize()
        keep = (cell >= 0) & (cell < nx * ny)
        n = int(cnt_out.item())
        assert n == int(keep.sum())
        st = starts.cpu().numpy()
        assert st[nt] == n and np.all(st[nt + 1:] == -7)
        got = _arrays(dst[d_off:d_off + nbytes], cap, 2, n)
        assert np.array_equal(np.sort(got["id"]), ids[keep])
        assert np.all(np.diff(_tile_key(got["cell"], nx, ny, tile, 2)) >= 0)
        # the guard bytes after dst are untouched
        assert bool(torch.all(dst[d_off + nbytes:d_off + nbytes + guard] == 0xA5))
    # the shared scratch still serves a normal call afterwards
    cnt_in.fill_(cap // 2)
    rc = L.lpic_sort_tiles_static(2, nx, ny, 1, t3, src.data_ptr() + s_off, dst.data_ptr() + d_off,
                                  cap, cnt_in.data_ptr(), cnt_out.data_ptr(), starts.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    keep = (cell[:cap // 2] >= 0) & (cell[:cap // 2] < nx * ny)
    assert int(cnt_out.item()) == int(keep.sum())
