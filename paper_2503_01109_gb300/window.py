"""Batched keyframe window: all views' forward, loss and adjoint in one persistent
launch (``fgs_render_window``), plus the tile-size / batch-depth autotuner.

A window iteration is: project every Gaussian into every view, bin and sort all
views at once, the persistent render-loss-adjoint launch, the projection adjoint,
eq15, Adam.  It allocates and synchronises nothing, so it is captured into a CUDA
graph and replayed (:meth:`Window.capture`).
"""
from __future__ import annotations

import torch

from . import fgs
from .mapping import Mapper, PAPER_LOSS, PAPER_REG


class Window(Mapper):
    def __init__(self, g: fgs.GaussianMap, cams: list, til: fgs.Tiling | None = None, **kw):
        kw.setdefault("use_device_count", True)
        super().__init__(g, cams, til, **kw)
        self.ws_win = fgs.ws_tensor(fgs.fgs_render_window_workspace_size(self.cams), g.buf.device)
        self.graph = None

    def iteration(self):
        fgs.fgs_project(self.g, self.cams, self.til, self.proj, self.status, self.use_dc)
        n = self.g.capacity if self.use_dc else self.g.n
        fgs.fgs_bin_sort(self.proj, n, self.cams, self.til, self.ws_bin, self.tile_keys, self.ids, self.ranges,
                         self.num_pairs, self.status, d_n=self.g.d_n if self.use_dc else None)
        if self.fused_tail:
            self.ensure_clean()
        else:
            fgs.fgs_memset_async(self.grads.buf)
            fgs.fgs_memset_async(self.grad2d)
        fgs.fgs_memset_async(self.loss_acc)
        fgs.fgs_render_window(self.g, self.proj, self.cams, self.til, self.ids, self.ranges, self.color_gt,
                              self.depth_gt, *self.loss_w, self.frame, self.dC, self.dD, self.grad2d, self.grads,
                              self.loss_acc, self.ws_win, self.status, self.use_dc, tile_order=self.tile_order)
        self._order()   # heaviest first for the next window iteration
        if self.fused_tail:
            self.fused_tail_step()
            return
        fgs.fgs_project_bwd(self.g, self.proj, self.cams, self.grad2d, self.grads, self.use_dc)
        if self.reg_w != 0.0:
            fgs.fgs_scale_reg(self.g, self.reg_w, self.grads, self.loss_acc, self.ws_reg, self.use_dc)
        self.host_step += 1
        fgs.fgs_adam(self.g, self.grads, self.m, self.v, self.lr, step=self.host_step,
                     d_step=self.d_step if self.use_dc else None, use_device_count=self.use_dc)

    def capture(self, warmup: int = 2):
        """Capture one iteration into a CUDA graph (after `warmup` eager ones)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.iteration()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.iteration()
        return self.graph

    def replay(self):
        self.graph.replay()


def autotune(g: fgs.GaussianMap, cams, color_gt, depth_gt, reps: int = 5, loss_w=PAPER_LOSS,
             pair_capacity: int | None = None, use_device_count: bool = True):
    """The library's tiling autotuner (``fgs_autotune``) on this window: times every
    tile shape x batch depth (projection, binning, the persistent launch and the
    projection adjoint; the map is only read) and returns (best tiling,
    {(tile, batch): ms per pass})."""
    if pair_capacity is None:
        pair_capacity = min(2 ** 31 - 1, max(1 << 20, 64 * g.capacity * len(cams)))
    ws = fgs.ws_tensor(fgs.fgs_autotune_workspace_size(g, cams, pair_capacity, use_device_count), g.buf.device)
    best, ms = fgs.fgs_autotune(g, cams, color_gt, depth_gt, *loss_w, pair_capacity, reps, ws, use_device_count)
    del ws
    return best, dict(zip(fgs.AUTOTUNE_ORDER, ms))


class KeyframeSelector:
    """The keyframe window of Sec. III-C: keyframes whose co-visibility with the
    current frame exceeds `threshold` (co-visible) plus a random `frac` of the
    others, decided on the device (``fgs_covisibility``, ``fgs_select_keyframes``);
    the uniform draws come from a seeded generator.  At most `max_keyframes` are
    returned: co-visible ones by decreasing co-visibility, then random ones in draw
    order."""

    def __init__(self, step: int = 4, threshold: float = 0.7, frac: float = 0.3, seed: int = 0,
                 max_keyframes: int = 7, device="cuda"):
        self.step, self.threshold, self.frac, self.max_k = int(step), float(threshold), float(frac), max_keyframes
        self.gen = torch.Generator(device="cpu").manual_seed(seed)
        self.device = device
        self.valid = torch.zeros(1, dtype=torch.int64, device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)

    def select(self, depth: torch.Tensor, cam: dict, keyframes: list) -> list:
        K = len(keyframes)
        if K == 0:
            return []
        inside = torch.zeros(K, dtype=torch.int64, device=self.device)
        kind = torch.zeros(K, dtype=torch.int32, device=self.device)
        u = torch.rand(K, generator=self.gen).to(self.device)
        for a in range(0, K, 256):  # at most 256 keyframes per co-visibility call
            fgs.fgs_covisibility(depth, cam, keyframes[a:a + 256], self.step, inside[a:a + 256], self.valid)
        fgs.fgs_select_keyframes(inside, self.valid, u, self.threshold, self.frac, kind, self.count)
        kind_h, inside_h, u_h = kind.cpu().numpy(), inside.cpu().numpy(), u.cpu().numpy()
        covis = sorted((k for k in range(K) if kind_h[k] == 1), key=lambda k: (-int(inside_h[k]), k))
        rand = sorted((k for k in range(K) if kind_h[k] == 2), key=lambda k: (float(u_h[k]), k))
        return (covis + rand)[:self.max_k]
