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
    # two allocation-free calls back to back on the shared scratch array, the
    # larger view set first: stale partial sums of the first call would show up in
    # the second call's loss if they were read.  Both entry points run the same
    # kernels and reduce the partials in one fixed order, so the results are equal
    # bit for bit.
    runs = [([syn.pinhole(1200, 680, 600.0), syn.pinhole(70, 45, 60.0)], 3, (0.9, 0.1, 0.1)),
            ([syn.pinhole(64, 48, 60.0)], 4, (1.0, 1.0, 0.0))]
    imgs = [_images(cams, seed) for cams, seed, _ in runs]
    got = [_without_workspace(cams, im, w) for (cams, _, w), im in zip(runs, imgs)]
    torch.cuda.synchronize()
    ref = [_with_workspace(cams, im, w) for (cams, _, w), im in zip(runs, imgs)]
    torch.cuda.synchronize()
    for g, r in zip(got, ref):
        for a, b in zip(g, r):
            assert torch.equal(a, b)
    assert float(got[1][0].item()) != float(got[0][0].item())


def test_noalloc_loss_rejects_view_sets_beyond_its_scratch():
    cams = [syn.pinhole(4096, 4096, 1000.0)] * 8      # 8 x 16384 loss tiles (32x32 px) > 65536
    dummy = torch.zeros(16, device="cuda")
    p = fgs.LossParams(0.9, 0.1, 0.1)
    rc = fgs.lib().fgs_loss_noalloc(fgs.camera_array(cams), len(cams), fgs._ptr(dummy), fgs._ptr(dummy),
                                    fgs._ptr(dummy), fgs._ptr(dummy), ctypes.byref(p), fgs._ptr(dummy),
                                    fgs._ptr(dummy), fgs._ptr(dummy), None)
    assert rc == 3 and b"scratch" in fgs.lib().fgs_last_error()


def test_noalloc_loss_errors_name_the_entry_point():
    dummy = torch.zeros(16, device="cuda")
    p = fgs.LossParams(0.9, 0.1, 0.1)
    rc = fgs.lib().fgs_loss_noalloc(fgs.camera_array([syn.pinhole(8, 8, 8.0)]), 0, fgs._ptr(dummy), fgs._ptr(dummy),
                                    fgs._ptr(dummy), fgs._ptr(dummy), ctypes.byref(p), fgs._ptr(dummy),
                                    fgs._ptr(dummy), fgs._ptr(dummy), None)
    assert rc == 1 and fgs.lib().fgs_last_error().startswith(b"fgs_loss_noalloc:")
