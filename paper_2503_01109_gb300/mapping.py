"""The dense-map mapping iteration (Sec. III-D) on top of the C ABI.

:class:`Mapper` owns every buffer of one view set (projection records, pair
lists, render outputs, gradients, Adam moments, workspaces) so that an
iteration -- project, bin and sort, blend (eq1), loss (eq16 with eq15), adjoint,
Adam -- launches library kernels only, allocates nothing and synchronises
nothing.  With ``use_device_count`` the live Gaussian count stays on the device
(seeding can append without a host round trip) and the iteration can be captured
into a CUDA graph and replayed.

:class:`RenderFn` is the differentiable render behind ``torch.autograd``: its
backward is the library's hand-written adjoint (``fgs_render_bwd``).
"""
from __future__ import annotations

import torch

from . import fgs

# eq16 weights (lambda_i, lambda_d, 1 - lambda_i) and eq15 weight (lambda_r); the
# paper does not state them.
PAPER_LOSS = (0.9, 0.1, 0.1)
PAPER_REG = 0.01


class Mapper:
    def __init__(self, g: fgs.GaussianMap, cams: list, til: fgs.Tiling | None = None, pair_capacity: int | None = None,
                 loss_w=PAPER_LOSS, reg_w: float = PAPER_REG, lr=fgs.DEFAULT_LR, use_device_count: bool = True,
                 fused_tail: bool = True, keep_tile_keys: bool = True):
        dev = g.buf.device
        self.g, self.cams = g, list(cams)
        self.til = til or fgs.tiling(16, 16, 128)
        self.V = len(cams)
        self.loss_w, self.reg_w, self.lr = tuple(loss_w), float(reg_w), tuple(lr)
        self.use_dc = use_device_count
        cap = g.capacity
        self.proj = fgs.Projection(self.V, cap, dev)
        self.frame = fgs.Frame(self.cams, dev)
        self.n_tiles = fgs.num_tiles(self.cams, self.til)
        if pair_capacity is None:
            pair_capacity = min(2 ** 31 - 1, max(1 << 20, 64 * cap * self.V))
        self.pair_capacity = int(pair_capacity)
        # the pairs' tile indices: redundant with `ranges`, kept for inspection
        self.tile_keys = torch.zeros(self.pair_capacity, dtype=torch.int32, device=dev) if keep_tile_keys else None
        self.ids = torch.zeros(self.pair_capacity, dtype=torch.int32, device=dev)
        self.ranges = torch.zeros(self.n_tiles, 2, dtype=torch.int32, device=dev)
        # launch order of the render kernels' tiles: heaviest first by the last
        # render's contributor counts (fgs_tile_order), any permutation being valid
        self.tile_order = torch.arange(self.n_tiles, dtype=torch.int32, device=dev)
        self.ws_order = fgs.ws_tensor(fgs.fgs_tile_order_workspace_size(self.cams, self.til), dev)
        self.num_pairs = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.ws_bin = fgs.ws_tensor(fgs.fgs_bin_sort_workspace_size(self.cams, self.til, self.V * cap,
                                                                    self.pair_capacity), dev)
        self.grad2d = torch.zeros(self.V, cap, 8, dtype=torch.float32, device=dev)
        self.grads = g.zeros_like()
        self.m = g.zeros_like()
        self.v = g.zeros_like()
        self.dC = torch.zeros_like(self.frame.color)
        self.dD = torch.zeros_like(self.frame.depth)
        self.loss_acc = torch.zeros(1, dtype=torch.float32, device=dev)
        self.ws_loss = fgs.ws_tensor(fgs.fgs_loss_workspace_size(self.cams), dev)
        self.ws_reg = fgs.ws_tensor(fgs.fgs_scale_reg_workspace_size(cap), dev)
        self.d_step = torch.zeros(1, dtype=torch.int32, device=dev)
        # the iteration's tail (projection adjoint, eq15, Adam) as one fused call that
        # leaves the RGB gradient and grad2d zero; `_clean` tracks that state
        self.fused_tail = bool(fused_tail)
        self.ws_fused = fgs.ws_tensor(fgs.fgs_project_bwd_adam_workspace_size(cap), dev)
        self._clean = True
        self.ws_prune = None
        self.num_kept = torch.zeros(1, dtype=torch.int64, device=dev)
        self.color_gt = torch.zeros_like(self.frame.color)
        self.depth_gt = torch.zeros_like(self.frame.depth)
        self.host_step = 0

    # ------------------------------------------------------------------------------
    def set_target(self, color_gt: torch.Tensor, depth_gt: torch.Tensor):
        self.color_gt.copy_(color_gt.reshape(-1))
        self.depth_gt.copy_(depth_gt.reshape(-1))

    def set_cameras(self, cams: list):
        assert len(cams) == self.V and all(c["width"] == o["width"] and c["height"] == o["height"]
                                          for c, o in zip(cams, self.cams))
        self.cams = list(cams)
        self.frame.cams = self.cams

    def render(self, sample_stride: int = 1):
        """a1-a5: project, bin + sort, blend (on every second pixel in x and y when
        sample_stride is 2; the other pixels get the background)."""
        fgs.fgs_project(self.g, self.cams, self.til, self.proj, self.status, self.use_dc)
        n = self.g.capacity if self.use_dc else self.g.n
        fgs.fgs_bin_sort(self.proj, n, self.cams, self.til, self.ws_bin, self.tile_keys, self.ids, self.ranges,
                         self.num_pairs, self.status, d_n=self.g.d_n if self.use_dc else None)
        self._blend(sample_stride)
        self._order()

    def _blend(self, sample_stride: int):
        if sample_stride == 1:
            fgs.fgs_render_fwd(self.proj, self.g, self.cams, self.til, self.ids, self.ranges, self.frame, self.status,
                               tile_order=self.tile_order)
        else:
            fgs.fgs_render_fwd_sampled(self.proj, self.g, self.cams, self.til, self.ids, self.ranges, self.frame,
                                       sample_stride, self.status, tile_order=self.tile_order)

    def _order(self):
        """The tiles heaviest first by this render's contributor counts: the order of
        the adjoint that follows and of the next render."""
        fgs.fgs_tile_order(self.cams, self.til, self.frame.n_contrib, self.tile_order, self.ws_order)

    def can_sample(self, stride: int) -> bool:
        """Whether render(sample_stride=stride) is available for this tiling."""
        return stride == 1 or (stride == 2 and self.til.tile_w == 16)

    def backward(self, dC, dD, dA=None):
        """a7-a8 into self.grads (cleared first)."""
        fgs.fgs_memset_async(self.grads.buf)
        fgs.fgs_render_bwd(self.g, self.proj, self.cams, self.til, self.ids, self.ranges, self.frame, dC, dD, dA,
                           self.grad2d, self.grads, self.status, self.use_dc, tile_order=self.tile_order)
        self._clean = False

    def ensure_clean(self):
        """Zeroes the RGB gradient and grad2d unless the last fused tail left them so."""
        if not self._clean:
            fgs.fgs_memset_async(self.grads.buf)
            fgs.fgs_memset_async(self.grad2d)
            self._clean = True

    def fused_tail_step(self):
        """a8 + eq15 + a9 in one pass per Gaussian (fgs_project_bwd_adam)."""
        self.host_step += 1
        fgs.fgs_project_bwd_adam(self.g, self.proj, self.cams, self.grad2d, self.grads, self.reg_w, self.loss_acc,
                                 self.m, self.v, self.lr, step=self.host_step,
                                 d_step=self.d_step if self.use_dc else None, ws=self.ws_fused,
                                 use_device_count=self.use_dc)
        self._clean = True

    def iteration(self):
        """One mapping iteration a1-a9 against the current target."""
        self.render()
        fgs.fgs_memset_async(self.loss_acc)
        fgs.fgs_loss(self.cams, self.frame.color, self.frame.depth, self.color_gt, self.depth_gt, *self.loss_w,
                     self.dC, self.dD, self.loss_acc, self.ws_loss)
        if self.fused_tail:
            self.ensure_clean()
            fgs.fgs_render_bwd_splats(self.g, self.proj, self.cams, self.til, self.ids, self.ranges, self.frame,
                                      self.dC, self.dD, None, self.grad2d, self.grads, self.status, self.use_dc,
                                      tile_order=self.tile_order)
            self.fused_tail_step()
            return
        self.backward(self.dC, self.dD)
        if self.reg_w != 0.0:
            fgs.fgs_scale_reg(self.g, self.reg_w, self.grads, self.loss_acc, self.ws_reg, self.use_dc)
        self.host_step += 1
        fgs.fgs_adam(self.g, self.grads, self.m, self.v, self.lr, step=self.host_step,
                     d_step=self.d_step if self.use_dc else None, use_device_count=self.use_dc)

    def prune(self, params: fgs.PruneParams):
        """Gaussian pruning (Sec. III-A): drops too large or nearly transparent
        Gaussians from the map and their Adam moments, keeping the others' order.
        With the device count nothing synchronises; otherwise the host count is
        read back."""
        if self.ws_prune is None:
            self.ws_prune = fgs.ws_tensor(fgs.fgs_prune_workspace_size(self.g.capacity), self.g.buf.device)
        fgs.fgs_prune(self.g, self.m, self.v, params, self.ws_prune, self.num_kept, self.use_dc)
        if not self.use_dc:
            self.g.n = int(self.num_kept.item())

    # ------------------------------------------------------------------------------
    def state_dict(self) -> dict:
        """The mapping state for checkpoint / resume (host tensors): the live Gaussians'
        parameters and both Adam moments, the live count and the step counters."""
        n = int(self.g.d_n.item()) if self.use_dc else self.g.n
        return {"n": n, "params": self.g.buf[:, :n].cpu(), "m": self.m.buf[:, :n].cpu(),
                "v": self.v.buf[:, :n].cpu(), "host_step": self.host_step, "d_step": int(self.d_step.item())}

    def load_state_dict(self, st: dict):
        """Restores a state_dict() into this mapper's buffers (same or larger capacity);
        gradients and per-pixel state start clean, as after a completed iteration."""
        n = int(st["n"])
        if n > self.g.capacity:
            raise ValueError(f"checkpoint holds {n} Gaussians, capacity is {self.g.capacity}")
        for gm, key in ((self.g, "params"), (self.m, "m"), (self.v, "v")):
            gm.buf.zero_()
            gm.buf[:, :n].copy_(st[key])
        for gm in (self.g, self.m, self.v, self.grads):
            gm.n = n
            gm.d_n.fill_(n)
        self.host_step = int(st["host_step"])
        self.d_step.fill_(int(st["d_step"]))
        self.grads.buf.zero_()
        self.grad2d.zero_()
        self._clean = True

    def check_status(self):
        s = int(self.status.item())
        if s:
            raise fgs.FGSError(f"device status {s} (pairs needed: {int(self.num_pairs.item())}, "
                               f"capacity {self.pair_capacity})")


class RenderFn(torch.autograd.Function):
    """(params [14][capacity]) -> (color, depth, alpha) of a view set, with the
    library's adjoint as backward.  ``ctx`` keeps the Mapper whose buffers hold
    the forward's lists and per-pixel state."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, mapper: Mapper):
        assert params.data_ptr() == mapper.g.buf.data_ptr(), "params must be the mapper's Gaussian buffer"
        mapper.render()
        ctx.mapper = mapper
        f = mapper.frame
        return f.color.clone(), f.depth.clone(), f.alpha.clone()

    @staticmethod
    def backward(ctx, dC, dD, dA):
        m = ctx.mapper
        z = torch.zeros_like(m.frame.depth)
        m.backward(dC.contiguous() if dC is not None else torch.zeros_like(m.frame.color),
                   dD.contiguous() if dD is not None else z, dA.contiguous() if dA is not None else None)
        return m.grads.buf.clone(), None


def render(params: torch.Tensor, mapper: Mapper):
    return RenderFn.apply(params, mapper)
