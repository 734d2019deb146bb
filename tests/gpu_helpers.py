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
