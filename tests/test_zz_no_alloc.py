"""fgs_loss_noalloc: the workspace-free variant of the loss for callers that may
not allocate device memory (a host that owns every device byte through its own
pool, or a real-time loop that cannot take cudaMalloc's latency).  It must give
the same loss and gradients as fgs_loss on back-to-back calls -- the scratch
array it keeps between calls must not leak one call's partial sums into the
next -- and refuse view sets beyond its fixed scratch size.

This file is collected last on purpose; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_01109_gb300 import fgs, synthetic as syn

pytestmark = pytest.mark.gpu


def _images(cams, seed):
    rng = np.random.default_rng(seed)
    Cs = [rng.uniform(0, 1, (3, c["height"], c["width"])) for c in cams]
    Cg = [rng.uniform(0, 1, (3, c["height"], c["width"])) for c in cams]
    Ds = [rng.uniform(1, 3, (c["height"], c["width"])) for c in cams]
    Dg = [rng.uniform(1, 3, (c["height"], c["width"])) * (rng.uniform(0, 1, (c["height"], c["width"])) > 0.1)
          for c in cams]
    color, depth = fgs.pack_images(cams, Cs, Ds)
    color_gt, depth_gt = fgs.pack_images(cams, Cg, Dg)
    return color, depth, color_gt, depth_gt


def _with_workspace(cams, imgs, w):
    color, depth, color_gt, depth_gt = imgs
    dC, dD = torch.zeros_like(color), torch.zeros_like(depth)
    acc = torch.zeros(1, device="cuda")
    ws = fgs.ws_tensor(fgs.fgs_loss_workspace_size(cams))
    fgs.fgs_loss(cams, color, depth, color_gt, depth_gt, *w, dC, dD, acc, ws)
    return acc, dC, dD


def _without_workspace(cams, imgs, w):
    color, depth, color_gt, depth_gt = imgs
    dC, dD = torch.zeros_like(color), torch.zeros_like(depth)
    acc = torch.zeros(1, device="cuda")
    fgs.fgs_loss_noalloc(cams, color, depth, color_gt, depth_gt, *w, dC, dD, acc)
    return acc, dC, dD


def test_noalloc_loss_matches_workspace_loss_twice_in_a_row():
    assert torch.cuda.is_available()
    # two different view sets back to back: the second call is smaller, so stale
    # partials of the first would show up in its sum if they were read
    runs = [([syn.pinhole(1200, 680, 600.0), syn.pinhole(70, 45, 60.0)], 3, (0.9, 0.1, 0.1)),
            ([syn.pinhole(64, 48, 60.0)], 4, (1.0, 1.0, 0.0))]
    for cams, seed, w in runs:
        imgs = _images(cams, seed)
        ref = _with_workspace(cams, imgs, w)
        got = _without_workspace(cams, imgs, w)
        torch.cuda.synchronize()
        assert float(got[0].item()) == pytest.approx(float(ref[0].item()), rel=1e-5)
        for a, b in zip(got[1:], ref[1:]):
            assert torch.allclose(a, b, rtol=0, atol=1e-4 * float(b.abs().max().item()))


def test_noalloc_loss_rejects_view_sets_beyond_its_scratch():
    cams = [syn.pinhole(4096, 4096, 1000.0)] * 2      # 2 x 65536 loss tiles > 65536
    dummy = torch.zeros(16, device="cuda")
    p = fgs.LossParams(0.9, 0.1, 0.1)
    rc = fgs.lib().fgs_loss_noalloc(fgs.camera_array(cams), len(cams), fgs._ptr(dummy), fgs._ptr(dummy),
                                    fgs._ptr(dummy), fgs._ptr(dummy), ctypes.byref(p), fgs._ptr(dummy),
                                    fgs._ptr(dummy), fgs._ptr(dummy), None)
    assert rc == 3 and b"scratch" in fgs.lib().fgs_last_error()
