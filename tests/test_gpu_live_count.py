"""A map whose Gaussian count stays on the device (d_n): fgs_project writes full
records for the live slots only and radius 0 past them, and fgs_bin_sort with d_n
bins the live slots only.  The lists equal those of binning every slot without
d_n, and the oracle's lists over the live Gaussians (teacher-forced on the GPU's
float32 records), bit for bit; a live count of zero gives no pairs."""
import numpy as np
import pytest
import torch

from oracle import render as orr
from paper_2503_01109_gb300 import fgs, synthetic as syn

from gpu_helpers import make_mapper

pytestmark = pytest.mark.gpu


def _lists(m, d_n):
    fgs.fgs_bin_sort(m.proj, m.g.capacity, m.cams, m.til, m.ws_bin, m.tile_keys, m.ids, m.ranges, m.num_pairs,
                     m.status, d_n=d_n)
    torch.cuda.synchronize()
    P = int(m.num_pairs.item())
    return m.tile_keys[:P].cpu().numpy().copy(), m.ids[:P].cpu().numpy().copy(), m.ranges.cpu().numpy().copy()


@pytest.mark.parametrize("live_frac", [0.6, 1.0, 0.0])
def test_live_slots_only(cuda_device, live_frac):
    n = 4000
    sc = syn.tiny_scene(n, seed=5)
    cams = [syn.pinhole(96, 64, 70.0), syn.pinhole(40, 30, 45.0, syn.look_pose([0.05, -0.02, 0.1], 0.08, 0.02))]
    m = make_mapper(sc, cams, (16, 16), 64, capacity=2 * n, use_dc=True)
    # fill the records of every slot first (a larger live count), then lower it:
    # the slots past the new count keep stale splats and rects
    fgs.fgs_project(m.g, m.cams, m.til, m.proj, m.status, True)
    live = int(live_frac * n)
    m.g.d_n.fill_(live)
    fgs.fgs_project(m.g, m.cams, m.til, m.proj, m.status, True)
    torch.cuda.synchronize()
    assert int(m.status.item()) == 0
    V = len(cams)
    assert not m.proj.radius[:, live:].any()                     # past the live count: radius 0
    got = _lists(m, m.g.d_n)
    every = _lists(m, None)
    for a, b in zip(got, every):
        assert np.array_equal(a, b)
    if live == 0:
        assert len(got[0]) == 0 and not got[2].any()
        return
    depth = np.stack([m.proj.splat[v, :live, 6].cpu().numpy() for v in range(V)]).astype(np.float32)
    radius = np.stack([m.proj.radius[v, :live].cpu().numpy() for v in range(V)])
    rect = np.stack([m.proj.rect[v, :live].cpu().numpy().view(np.uint16).astype(np.int32) for v in range(V)])
    supp = np.stack([orr.support_f32(m.proj.splat[v, :live].cpu().numpy()) for v in range(V)])
    rt, rids, rranges = orr.bin_sort(cams, 16, 16, depth, radius, rect, supp)
    assert len(rt) > 1000
    assert np.array_equal(got[0], rt) and np.array_equal(got[1], rids) and np.array_equal(got[2], rranges)
