"""Shared set-up of the GPU parity tests: scenes on the device, render through
the C ABI, and the oracle comparisons (tolerances from the parity contract:
bit-exact key lists, 1e-4 absolute per pixel, 1e-3 relative gradients)."""
from __future__ import annotations

import numpy as np
import torch

from oracle import render as orr
from paper_2503_01109_gb300 import fgs, synthetic as syn
from paper_2503_01109_gb300.mapping import Mapper

PIX_TOL = 1e-4
GRAD_REL = 1e-3


def make_mapper(scene, cams, tile=(16, 16), batch=128, capacity=None, use_dc=False, **kw):
    g = fgs.GaussianMap.from_scene(scene, capacity)
    m = Mapper(g, cams, fgs.tiling(tile[0], tile[1], batch), use_device_count=use_dc, **kw)
    return m


def gpu_lists(m: Mapper):
    P = int(m.num_pairs.item())
    assert int(m.status.item()) == 0, "device status set"
    return (m.tile_keys[:P].cpu().numpy().view(np.uint32), m.ids[:P].cpu().numpy(), m.ranges.cpu().numpy())


def gpu_view_splats(m: Mapper, v: int, n: int):
    s = m.proj.splat[v, :n].cpu().numpy()
    r = m.proj.radius[v, :n].cpu().numpy()
    rc = m.proj.rect[v, :n].cpu().numpy().view(np.uint16).astype(np.int32)
    # empty rect is stored as x0 = y0 = 1, x1 = y1 = 0
    return orr.splats_from_gpu(s, r, rc), s


def grad_close(g, ref, rel=GRAD_REL):
    """|g - g*| <= rel * max(|g*|, 1e-3 * max|g*|) elementwise."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    floor = 1e-3 * np.abs(ref).max() if ref.size else 0.0
    bound = rel * np.maximum(np.abs(ref), floor) + 1e-30
    bad = np.abs(g - ref) > bound
    return bad, np.abs(g - ref) / np.maximum(np.abs(ref), floor + 1e-30)


def tile_origin(cams, tw, th):
    out, base = [], 0
    for c in cams:
        tx, ty = orr.tiles_of(c, tw, th)
        out.append(base)
        base += tx * ty
    return out


GRAD_KEYS = ("means", "log_scales", "quats", "logits", "rgb")


def oracle_flags(m: Mapper, cams, n: int, rgb_aos: np.ndarray, tw: int, th: int):
    """Per-view decision-band flags [H][W] (bool) of the teacher-forced forward:
    the oracle's FP64 blend of the GPU's float32 splats over the GPU's lists marks
    every pixel where a float32 evaluation could take the other branch of a
    threshold decision (alpha vs 1/255 or 0.99, T vs 1e-4, power vs 0)."""
    _, ids, ranges = gpu_lists(m)
    bases = tile_origin(cams, tw, th)
    out = []
    for v, cam in enumerate(cams):
        gsp, _ = gpu_view_splats(m, v, n)
        out.append(orr.render_fwd(gsp, rgb_aos, cam, ids, ranges, bases[v], tw, th)["flag"] != 0)
    return out


def masked(images, flags):
    """Per-view image arrays ([3][H][W] or [H][W]) with the flagged pixels set to
    zero: an upstream gradient masked this way on both sides removes the flagged
    pixels' terms from every parameter gradient."""
    out = []
    for img, f in zip(images, flags):
        a = np.array(img, np.float32, copy=True)
        a[..., f] = 0.0
        out.append(a)
    return out


def to_device(images):
    return torch.cat([torch.as_tensor(np.ascontiguousarray(x)).reshape(-1) for x in images]).cuda()


def assert_grads_exact(grads_gpu: fgs.GaussianMap, ref: dict, n: int, rel: float = GRAD_REL, keys=GRAD_KEYS):
    """Every entry of every gradient plane within |g - g*| <= rel max(|g*|, 1e-3 max|g*|)."""
    for key in keys:
        got = grads_gpu.plane(key)[:, :n].cpu().numpy().reshape(ref[key].shape)
        bad, r = grad_close(got, ref[key], rel)
        assert not bad.any(), (key, int(bad.sum()), float(r.max()))


def flag_fraction(flags) -> float:
    tot = sum(f.size for f in flags)
    return sum(int(f.sum()) for f in flags) / max(tot, 1)
