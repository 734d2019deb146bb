"""The per-frame pipeline the benchmark times (FramePipeline.frame_step): render at
the frame's pose on the seed grid, Fourier seeding whose frame-only half runs on
a second stream, three mapping iterations in the heaviest-first tile order, and
pruning.  With the overlap the first frame's seeds are those of the one-call
seeding bit for bit, and later frames keep the status clear and the loss finite,
from resident frames and from pinned host buffers."""
import numpy as np
import pytest
import torch

from paper_2503_01109_gb300 import synthetic as syn
from paper_2503_01109_gb300.frames import FramePipeline

pytestmark = pytest.mark.gpu

W, H, F = 256, 160, 200.0


def _pipeline(overlap: bool):
    cams = syn.trajectory(4, seed=7, width=W, height=H, f=F)
    scene = syn.room_scene(30_000, seed=1, kind="map")
    gt = syn.room_scene(60_000, seed=2, kind="gt")
    return FramePipeline(scene, cams, gt, capacity=30_000 + 5 * 50_000, overlap_seeding=overlap, device="cuda")


def test_overlapped_seeding_matches_the_one_call_seeding(cuda_device):
    runs = {}
    for overlap in (False, True):
        p = _pipeline(overlap)
        n0 = p.live_count()
        p.frame_step(0)
        torch.cuda.synchronize()
        p.check()
        k = int(p.seeder.num_new.item())
        assert k > 0
        runs[overlap] = (n0, k, p.seeder.seed_xy[:k].cpu().numpy(), p.seeder.mask.cpu().numpy(),
                         p.seeder.energy.cpu().numpy(), int(p.seeder.threshold.item()))
    a, b = runs[False], runs[True]
    assert a[0] == b[0] and a[1] == b[1] and a[5] == b[5]
    for x, y in zip(a[2:5], b[2:5]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("from_host", [False, True])
def test_frame_steps_keep_the_status_clear(cuda_device, from_host):
    p = _pipeline(True)
    hosts = [(c.cpu().pin_memory(), d.cpu().pin_memory()) for c, d in zip(p.colors, p.depths)] if from_host else None
    counts = []
    for k in range(4):
        p.frame_step(k, from_host=hosts[k] if hosts else None)
        torch.cuda.synchronize()
        p.check()
        counts.append(p.live_count())
        assert np.isfinite(float(p.mapper.loss_acc.item()))
    assert all(0 < c <= p.g.capacity for c in counts)
