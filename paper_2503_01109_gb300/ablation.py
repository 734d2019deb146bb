"""The densification ablation of the paper's tab6 on synthetic frames: equidistant
seeding (sparse or dense grid, large or small Gaussians) against the adaptive
Fourier densification of Sec. III-A, from an empty map with the same mapping
budget.

Equidistant seeding is the same seeding call with the two grids and the two
scale factors made equal (m = n, alpha_h = alpha_l), so the frequency mask no
longer changes where or how large the seeds are; the adaptive variant uses the
readings m = 2, alpha_h = 1 (high frequency) and n = 8, alpha_l = 4 (low).
Reported per variant: PSNR and SSIM of the final map over every frame (SSIM from
the library's own eq16 kernel with only its SSIM term), the Gaussian count and
the memory of their parameters and Adam moments.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fgs
from .convergence import SlamLoop

VARIANTS = {
    "sparse_equidistant_large": dict(m=8, n=8, alpha_h=4.0, alpha_l=4.0),
    "sparse_equidistant_small": dict(m=8, n=8, alpha_h=1.0, alpha_l=1.0),
    "dense_equidistant_large": dict(m=2, n=2, alpha_h=4.0, alpha_l=4.0),
    "dense_equidistant_small": dict(m=2, n=2, alpha_h=1.0, alpha_l=1.0),
    "adaptive": dict(m=2, n=8, alpha_h=1.0, alpha_l=4.0),
}


def ssim_all(loop: SlamLoop) -> float:
    """Mean SSIM of the final map over every frame: 1 - the SSIM-only eq16 loss."""
    m = loop.mapper
    vals = []
    ws = fgs.ws_tensor(fgs.fgs_loss_workspace_size([loop.cams[0]]), m.g.buf.device)
    acc = torch.zeros(1, dtype=torch.float32, device=m.g.buf.device)
    for k, cam in enumerate(loop.cams):
        m.set_cameras([cam])
        m.render()
        acc.zero_()
        fgs.fgs_loss([cam], m.frame.color, m.frame.depth, loop.colors[k], loop.depths[k], 0.0, 0.0, 1.0, m.dC, m.dD,
                     acc, ws)
        vals.append(1.0 - float(acc.item()))
    return float(np.mean(vals))


def densification_ablation(colors, depths, cams, capacity: int, iters_per_frame: int = 20, max_new: int = 400_000):
    out = {}
    for name, v in VARIANTS.items():
        sp = fgs.seed_params(max_new=max_new, **v)
        L = SlamLoop(colors, depths, cams, capacity, target_psnr=1e9, max_iters=iters_per_frame, seed_params=sp)
        L.run()
        n = int(L.g.d_n.item())
        out[name] = {"psnr_all_frames": L.evaluate_all(), "ssim_all_frames": ssim_all(L), "gaussians": n,
                     "memory_mb": n * 14 * 4 * 3 / 1e6, "seconds": float(sum(f["seconds"] for f in L.frames))}
    out["setup"] = (f"empty map, {len(cams)} frames, {iters_per_frame} mapping iterations per frame, up to "
                    f"{max_new} seeds per frame; memory = parameters + two Adam moments (14 floats each)")
    return out
