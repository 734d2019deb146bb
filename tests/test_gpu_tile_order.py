"""The launch order of the render kernels' tiles (fgs_tile_order): a permutation of
the view set's tiles sorted by each tile's largest contributor count (capped at
4095), heaviest first; renders launched in any order equal renders launched in
tile order; an order entry outside the tiles is skipped and reported."""
import numpy as np
import pytest
import torch

from gpu_helpers import grad_close, make_mapper
from paper_2503_01109_gb300 import fgs, synthetic as syn

pytestmark = pytest.mark.gpu

KEY_CAP = 4095
FIELDS = ("color", "depth", "alpha", "t_final", "n_contrib")
FGS_DEV_BAD_ORDER = 32


def tile_keys(ncs, cams, tw, th):
    """Per tile of the view set (views in order, tiles row-major): the largest
    contributor count of its pixels, capped."""
    keys = []
    for nc, c in zip(ncs, cams):
        H, W = c["height"], c["width"]
        ty, tx = -(-H // th), -(-W // tw)
        pad = np.zeros((ty * th, tx * tw), np.int64)
        pad[:H, :W] = nc
        keys.append(pad.reshape(ty, th, tx, tw).max(axis=(1, 3)).reshape(-1))
    return np.minimum(np.concatenate(keys), KEY_CAP)


@pytest.mark.parametrize("sizes, tile", [
    ([(1200, 680)], (16, 16)),                      # the benchmark frame's tiling
    ([(97, 61), (200, 131), (33, 20)], (16, 16)),   # ragged tiles in three views
    ([(200, 131), (64, 48)], (8, 8)),
    ([(300, 170)], (16, 32)),
])
def test_order_is_the_tiles_heaviest_first(cuda_device, sizes, tile):
    rng = np.random.default_rng(sum(w for w, _ in sizes) + tile[1])
    cams = [syn.pinhole(w, h, 0.8 * w) for w, h in sizes]
    til = fgs.tiling(*tile, 128)
    T = fgs.num_tiles(cams, til)
    ncs = []
    for w, h in sizes:
        nc = rng.geometric(1 / 300, (h, w)).astype(np.int64)
        nc[rng.random((h, w)) < 0.3] = 0                     # empty pixels, whole empty tiles below
        nc[: h // 3, : w // 4] = 0
        nc.flat[rng.integers(0, h * w, 3)] = rng.integers(KEY_CAP, 10 ** 6, 3)  # past the key cap
        ncs.append(nc.astype(np.int32))
    nc_dev = torch.from_numpy(np.concatenate([a.reshape(-1) for a in ncs])).cuda()
    order = torch.full((T,), -1, dtype=torch.int32, device="cuda")
    ws = fgs.ws_tensor(fgs.fgs_tile_order_workspace_size(cams, til))
    fgs.fgs_tile_order(cams, til, nc_dev, order, ws)
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(T))          # a permutation
    keys = tile_keys(ncs, cams, *tile)
    assert (keys == KEY_CAP).any() and (keys == 0).any()
    assert np.all(np.diff(keys[o]) <= 0)                     # heaviest first


def _frame(m):
    return {k: getattr(m.frame, k).cpu().numpy().copy() for k in FIELDS}


def _splat_grads(m, order):
    fgs.fgs_memset_async(m.grads.buf)
    fgs.fgs_memset_async(m.grad2d)
    fgs.fgs_render_bwd_splats(m.g, m.proj, m.cams, m.til, m.ids, m.ranges, m.frame, m.dC, m.dD, None, m.grad2d,
                              m.grads, m.status, False, tile_order=order)
    torch.cuda.synchronize()
    n = m.g.n
    return m.grad2d[:, :n].cpu().numpy().copy(), m.grads.buf[:, :n].cpu().numpy().copy()


@pytest.mark.parametrize("tile, batch", [((16, 16), 128), ((8, 8), 64), ((16, 32), 256)])
def test_renders_in_any_order_equal_the_tile_order(cuda_device, tile, batch):
    sc = syn.room_scene(60_000, seed=3)
    cams = [syn.room_camera(320, 200, 250.0, seed=4), syn.room_camera(97, 61, 80.0, seed=5)]
    m = make_mapper(sc, cams, tile, batch)
    m.render()
    torch.cuda.synchronize()
    heavy = m.tile_order.clone()
    rng = np.random.default_rng(1)
    shuffled = torch.from_numpy(rng.permutation(m.n_tiles).astype(np.int32)).cuda()
    torch.manual_seed(0)
    m.dC.copy_(torch.randn_like(m.dC))
    m.dD.copy_(torch.randn_like(m.dD))
    ref = None
    for order in (None, heavy, shuffled):
        for k in FIELDS:
            getattr(m.frame, k).zero_()
        fgs.fgs_render_fwd(m.proj, m.g, m.cams, m.til, m.ids, m.ranges, m.frame, m.status, tile_order=order)
        torch.cuda.synchronize()
        out = _frame(m)
        g2d, grgb = _splat_grads(m, order)
        if ref is None:
            ref = (out, g2d, grgb)
            assert (out["n_contrib"] > 0).mean() > 0.3
            continue
        for k in FIELDS:
            assert np.array_equal(out[k], ref[0][k]), k   # a tile's pixels do not depend on the order
        # the adjoint sums with float atomics, whose order follows the launch order
        for got, want in ((g2d, ref[1]), (grgb, ref[2])):
            bad, _ = grad_close(got, want, rel=1e-4)
            assert not bad.any()
    assert int(m.status.item()) == 0


def test_an_order_entry_outside_the_tiles_is_reported(cuda_device):
    sc = syn.room_scene(20_000, seed=3)
    cams = [syn.room_camera(200, 131, 160.0, seed=4)]
    m = make_mapper(sc, cams, (16, 16), 128)
    m.render()
    torch.cuda.synchronize()
    assert int(m.status.item()) == 0
    good = _frame(m)
    bad = torch.arange(m.n_tiles, dtype=torch.int32, device="cuda")
    bad[3] = m.n_tiles        # one past the last tile
    bad[5] = -2
    for k in FIELDS:
        getattr(m.frame, k).fill_(7)
    fgs.fgs_render_fwd(m.proj, m.g, m.cams, m.til, m.ids, m.ranges, m.frame, m.status, tile_order=bad)
    torch.cuda.synchronize()
    assert int(m.status.item()) & FGS_DEV_BAD_ORDER
    got = _frame(m)
    # tiles 3 and 5 were not rendered, every other tile was
    tx = -(-200 // 16)
    skipped = np.zeros((131, 200), bool)
    for t in (3, 5):
        y, x = divmod(t, tx)
        skipped[16 * y:16 * y + 16, 16 * x:16 * x + 16] = True
    for k in FIELDS:
        a, b = good[k].reshape(-1, 131, 200), got[k].reshape(-1, 131, 200)
        assert np.array_equal(a[:, ~skipped], b[:, ~skipped]), k
        assert np.all(b[:, skipped] == 7), k
    m.status.zero_()
    _splat_grads(m, bad)
    assert int(m.status.item()) & FGS_DEV_BAD_ORDER


def test_window_reports_an_order_entry_outside_the_tiles(cuda_device):
    from paper_2503_01109_gb300.window import Window
    cams = [syn.pinhole(70, 45, 60.0), syn.pinhole(33, 20, 30.0)]
    til = fgs.tiling(16, 16, 128)
    win = Window(fgs.GaussianMap.from_scene(syn.tiny_scene(1500, seed=7)), cams, til, reg_w=0.0)
    fr = [syn.textured_frame(c["width"], c["height"], 3 + i) for i, c in enumerate(cams)]
    cg, dg = fgs.pack_images(cams, [f["rgb"] for f in fr], [f["depth"] for f in fr])
    fgs.fgs_project(win.g, cams, til, win.proj, win.status, True)
    fgs.fgs_bin_sort(win.proj, win.g.capacity, cams, til, win.ws_bin, win.tile_keys, win.ids, win.ranges,
                     win.num_pairs, win.status)
    bad = torch.arange(win.n_tiles, dtype=torch.int32, device="cuda")
    bad[1] = 1 << 20
    for t in (win.grads.buf, win.grad2d, win.loss_acc):
        fgs.fgs_memset_async(t)
    fgs.fgs_render_window(win.g, win.proj, cams, til, win.ids, win.ranges, cg, dg, 0.9, 0.1, 0.1, win.frame, win.dC,
                          win.dD, win.grad2d, win.grads, win.loss_acc, win.ws_win, win.status, tile_order=bad)
    torch.cuda.synchronize()
    assert int(win.status.item()) == FGS_DEV_BAD_ORDER
