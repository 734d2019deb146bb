"""Tracking on the sparse map by GICP (Sec. III-B, eq12-eq14), on top of the C ABI.

:class:`SparseMap` holds the sparse Gaussian map: one point per occupied voxel
(uniform downsampling in 3D), its grid index and its regularised surface
covariances.  A keyframe adds its observed points in voxels the map does not
occupy yet (optionally only those of a mask, as the paper filters the source
cloud by the missing-region mask).

:class:`Tracker` turns a depth frame into the source cloud (pixels sampled every
`step` px, camera coordinates, covariances from their own neighbours) and runs
GICP against the map from an initial pose; every step runs in the library's
kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fgs


def cam_pose_inverse(world_to_cam) -> np.ndarray:
    """[R | t] -> [R^T | -R^T t] (3 x 4, float64)."""
    M = np.asarray(world_to_cam, np.float64).reshape(3, 4)
    R, t = M[:, :3], M[:, 3]
    return np.hstack([R.T, (-R.T @ t)[:, None]])


class SparseMap:
    def __init__(self, grid: fgs.Grid, voxel: fgs.Grid, capacity: int = 1 << 20, k: int = 10, eps: float = 1e-3,
                 device="cuda"):
        self.grid, self.voxel, self.k, self.eps = grid, voxel, int(k), float(eps)
        self.capacity = int(capacity)
        self.xyz = torch.zeros(self.capacity, 3, dtype=torch.float32, device=device)
        self.cov = torch.zeros(self.capacity, 6, dtype=torch.float32, device=device)
        self.n = torch.zeros(1, dtype=torch.int64, device=device)
        self.cell_start = torch.zeros(fgs.grid_cells(grid) + 1, dtype=torch.int32, device=device)
        self.order = torch.zeros(self.capacity, dtype=torch.int32, device=device)
        self.stage = torch.zeros(2 * self.capacity, 3, dtype=torch.float32, device=device)
        self.stage_n = torch.zeros(1, dtype=torch.int64, device=device)
        self.ws_grid = fgs.ws_tensor(fgs.fgs_grid_workspace_size(grid, self.capacity), device)
        self.ws_vox = fgs.ws_tensor(fgs.fgs_voxel_workspace_size(voxel, 2 * self.capacity), device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)

    def count(self) -> int:
        return int(self.n.item())

    def add(self, world_xyz: torch.Tensor, n_new: int):
        """Adds points [n_new][3] (world) in voxels the map does not occupy, then
        rebuilds the grid index and the covariances."""
        m = self.count()
        n_new = min(int(n_new), self.capacity)
        self.stage[:m].copy_(self.xyz[:m])
        self.stage[m:m + n_new].copy_(world_xyz[:n_new])
        self.stage_n.fill_(m + n_new)
        self.n.zero_()
        # the map's own points come first: one per voxel already, so all stay, in order
        fgs.fgs_voxel_downsample(self.stage, self.stage_n, self.voxel, self.ws_vox, self.xyz, self.n, self.status)
        fgs.fgs_grid_build(self.xyz, self.n, self.grid, self.cell_start, self.order, self.ws_grid)
        fgs.fgs_point_covariances(self.xyz, self.n, self.grid, self.cell_start, self.order, self.k, self.eps, self.cov)


class Tracker:
    def __init__(self, cam: dict, smap: SparseMap, src_grid: fgs.Grid, step: int = 8, iterations: int = 30,
                 max_dist: float = 0.1, overlap_dist: float = 0.05, device="cuda"):
        self.cam, self.map, self.src_grid, self.step = cam, smap, src_grid, int(step)
        W, H = cam["width"], cam["height"]
        cap = ((W + step - 1) // step) * ((H + step - 1) // step)
        self.src = torch.zeros(cap, 3, dtype=torch.float32, device=device)
        self.src_cov = torch.zeros(cap, 6, dtype=torch.float32, device=device)
        self.world = torch.zeros(cap, 3, dtype=torch.float32, device=device)
        self.n_src = torch.zeros(1, dtype=torch.int64, device=device)
        self.cell_start = torch.zeros(fgs.grid_cells(src_grid) + 1, dtype=torch.int32, device=device)
        self.order = torch.zeros(cap, dtype=torch.int32, device=device)
        self.ws_dp = fgs.ws_tensor(fgs.fgs_depth_points_workspace_size(W, H, step), device)
        self.ws_grid = fgs.ws_tensor(fgs.fgs_grid_workspace_size(src_grid, cap), device)
        self.ws_gicp = fgs.ws_tensor(fgs.fgs_gicp_workspace_size(cap), device)
        self.params = fgs.GicpParams(int(iterations), float(max_dist), float(overlap_dist))
        self.pose = torch.zeros(12, dtype=torch.float64, device=device)
        self.stats = torch.zeros(4, dtype=torch.float64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)

    def observe(self, depth: torch.Tensor, mask: torch.Tensor | None = None, mask_bits: int = 0xFF):
        """The source cloud of a depth frame and its covariances (camera frame)."""
        fgs.fgs_depth_points(depth, mask, mask_bits, self.cam, self.step, self.src, self.n_src, self.ws_dp,
                             self.status)
        fgs.fgs_grid_build(self.src, self.n_src, self.src_grid, self.cell_start, self.order, self.ws_grid)
        fgs.fgs_point_covariances(self.src, self.n_src, self.src_grid, self.cell_start, self.order, self.map.k,
                                  self.map.eps, self.src_cov)

    def track(self, pose0: np.ndarray):
        """GICP of the observed cloud against the map from pose0 (world-from-camera,
        3 x 4); returns (pose, stats: cost, pairs, overlap fraction, iterations)."""
        self.pose.copy_(torch.as_tensor(np.asarray(pose0, np.float64).reshape(-1)))
        m = self.map
        fgs.fgs_gicp(self.src, self.src_cov, self.n_src, m.xyz, m.cov, m.grid, m.cell_start, m.order, self.params,
                     self.pose, self.stats, self.ws_gicp)
        return self.pose.cpu().numpy().reshape(3, 4), self.stats.cpu().numpy()

    def add_keyframe(self, pose: np.ndarray):
        """Adds the observed cloud, placed at `pose`, to the sparse map."""
        self.pose.copy_(torch.as_tensor(np.asarray(pose, np.float64).reshape(-1)))
        fgs.fgs_transform_points(self.src, None, self.n_src, self.pose, self.world)
        self.map.add(self.world, int(self.n_src.item()))
