"""Fourier seeding of a frame into a map (Sec. III-A, eq2-eq11) on the device.

:class:`Seeder` owns the workspace, mask and counters for one image size and
calls ``fgs_fourier_seed`` with the map's render at the frame's pose (for the
missing-region check of eq9); new Gaussians are appended at the map's device
count, so no host synchronisation is needed.
"""
from __future__ import annotations

import torch

from . import fgs


class Seeder:
    def __init__(self, mapper, params: fgs.SeedParams | None = None, prior=None):
        if not hasattr(fgs.lib(), "fgs_fourier_seed"):
            raise AttributeError("fgs_fourier_seed missing from libfgs.so")
        cam = mapper.cams[0]
        W, H = int(cam["width"]), int(cam["height"])
        dev = mapper.g.buf.device
        self.mapper = mapper
        self.params = params or fgs.seed_params()
        self.prior = prior
        self.ws = fgs.ws_tensor(fgs.fgs_fourier_seed_workspace_size(W, H, self.params.max_new), dev)
        self.mask = torch.zeros(H * W, dtype=torch.uint8, device=dev)
        self.energy = torch.zeros(H * W, dtype=torch.float32, device=dev)
        self.num_new = torch.zeros(1, dtype=torch.int32, device=dev)
        self.seed_xy = torch.zeros(max(self.params.max_new, 1), 2, dtype=torch.int32, device=dev)
        self.threshold = torch.zeros(1, dtype=torch.int32, device=dev)

    def sample_stride(self) -> int:
        """2 when every seed pixel (the m- and n-grids of eq10) has even x and y and
        the tiling allows it: the render at the frame's pose is then needed there
        only (fgs_render_fwd_sampled), else 1."""
        p = self.params
        return 2 if (p.m % 2 == 0 and p.n % 2 == 0 and self.mapper.can_sample(2)) else 1

    def compute_energy(self, color_gt, cam: dict):
        """The first half of the seeding, which needs only the frame: the
        high-frequency energy E and its threshold (fgs_fourier_energy, eq2-eq8), on
        the current stream.  seed_frame(..., energy_stream=that stream) finishes
        it, so a caller can run this beside the render that seed_frame starts with."""
        fgs.fgs_fourier_energy(color_gt, cam, self.params, self.energy, self.threshold, self.ws)

    def seed_frame(self, color_gt, depth_gt, cam: dict, render_first: bool = True, first_frame: bool = False,
                   full_render: bool = False, energy_stream=None):
        """Render the map at `cam` (eq1 colour, depth, opacity) on the seed grid (every
        pixel when full_render or the grid is not even), then seed.  With
        energy_stream, compute_energy() was issued there for this frame: the seeds wait for
        it and reuse its E and threshold."""
        m = self.mapper
        m.set_cameras([cam])
        if render_first and not first_frame:
            m.render(1 if full_render else self.sample_stride())
        f = m.frame
        mlp = None if self.prior is None else self.prior.mlp_struct()
        if energy_stream is not None:
            torch.cuda.current_stream().wait_stream(energy_stream)
        fgs.fgs_fourier_seed(color_gt, depth_gt, None if first_frame else f.color, None if first_frame else f.depth,
                             None if first_frame else f.alpha, cam, self.params, mlp, self.mask, self.energy, m.g,
                             self.num_new, self.threshold, self.ws, m.status, use_device_count=True,
                             seed_xy=self.seed_xy, from_energy=energy_stream is not None)
