"""The seeding render on the sample grid (fgs_render_fwd_sampled): bit-identical to
the full render (fgs_render_fwd) on every pixel with even x and y, the background
everywhere else, and the Fourier seeding (Sec. III-A) fed by it appends exactly
the Gaussians it appends after a full render."""
import numpy as np
import pytest
import torch

from gpu_helpers import make_mapper
from paper_2503_01109_gb300 import fgs, frames, synthetic as syn
from paper_2503_01109_gb300.seeding import Seeder

pytestmark = pytest.mark.gpu

FIELDS = ("color", "depth", "alpha", "t_final", "n_contrib")


def _frame(m):
    return {k: getattr(m.frame, k).cpu().numpy().copy() for k in FIELDS}


@pytest.mark.parametrize("W,H,tile,batch,n", [
    (97, 61, (16, 16), 128, 20_000),       # odd sizes: the grid's last row / column, ragged tiles
    (200, 131, (16, 32), 64, 20_000),      # the tall tiling, another batch depth
    (1200, 680, (16, 16), 128, 300_000),   # a full frame
])
def test_sampled_render_equals_full_render_on_the_grid(cuda_device, W, H, tile, batch, n):
    sc = syn.room_scene(n, seed=3)
    cam = syn.room_camera(W, H, 0.5 * W, seed=4)
    m = make_mapper(sc, [cam], tile, batch)
    m.render(1)
    torch.cuda.synchronize()
    full = _frame(m)
    for k in FIELDS[:4]:                   # every pixel must be written by the sampled call
        getattr(m.frame, k).fill_(float("nan"))
    m.frame.n_contrib.fill_(-7)
    m.render(2)
    torch.cuda.synchronize()
    assert int(m.status.item()) == 0
    got = _frame(m)
    grid = np.zeros((H, W), bool)
    grid[::2, ::2] = True
    for k in FIELDS:
        a, b = full[k].reshape(-1, H, W), got[k].reshape(-1, H, W)
        assert np.array_equal(a[:, grid], b[:, grid]), k
        assert np.all(b[:, ~grid] == (1.0 if k == "t_final" else 0)), k
    assert (full["n_contrib"].reshape(H, W)[grid] > 0).mean() > 0.5   # the grid does see the map


def test_sampled_render_rejects_what_it_does_not_cover(cuda_device):
    sc = syn.room_scene(2000, seed=3)
    cam = syn.room_camera(64, 48, 40.0, seed=4)
    m = make_mapper(sc, [cam], (8, 8), 128)
    assert not m.can_sample(2)
    with pytest.raises(fgs.FGSError, match="16x16 or 16x32"):
        m.render(2)
    m16 = make_mapper(sc, [cam], (16, 16), 128)
    with pytest.raises(fgs.FGSError, match="sample_stride must be 2"):
        m16.render(3)


@pytest.mark.parametrize("grids", [dict(m=2, n=8), dict(m=4, n=4)])
def test_seeding_on_the_sampled_render_appends_the_same_gaussians(cuda_device, grids):
    W, H = 640, 480
    cam = syn.room_camera(W, H, 0.8 * W, seed=6)
    colors, depths = frames.render_targets(syn.room_scene(150_000, seed=8, kind="gt"), [cam])
    sc = syn.room_scene(60_000, seed=5)
    out = []
    for full in (True, False):
        m = make_mapper(sc, [cam], (16, 16), 128, capacity=60_000 + 100_000, use_dc=True)
        seeder = Seeder(m, fgs.seed_params(max_new=100_000, **grids))
        assert seeder.sample_stride() == 2
        seeder.seed_frame(colors[0], depths[0], cam, full_render=full)
        torch.cuda.synchronize()
        assert int(m.status.item()) == 0
        k = int(seeder.num_new.item())
        total = int(m.g.d_n.item())
        out.append((k, seeder.seed_xy[:k].cpu().numpy(), m.g.to_scene(total), seeder.mask.view(H, W).cpu().numpy()))
    (k0, xy0, g0, mask0), (k1, xy1, g1, mask1) = out
    assert k0 == k1 and k0 > 1000
    assert np.array_equal(xy0, xy1)
    for name in g0:
        assert np.array_equal(g0[name], g1[name]), name
    # M_h, M_l and the seeded bit everywhere; M_m (bit 2) wherever the sampled render blended
    assert np.array_equal(mask0 & 0b1011, mask1 & 0b1011)
    assert np.array_equal(mask0[::2, ::2], mask1[::2, ::2])
