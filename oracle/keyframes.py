"""Oracle of the keyframe co-visibility and window of Sec. III-C, "Keyframe
Selection" (test infrastructure only).

Co-visibility of a keyframe with the current frame: the fraction of the current
frame's observed points that fall inside the keyframe's view.  The observed
points are the current depth map sampled every `step` pixels from (0, 0), depth
> 0, back-projected through the current camera; a point is inside a keyframe when
it lies in front of its near plane and projects into its image (pixel centres at
integers, so the image spans [-0.5, W - 0.5) x [-0.5, H - 0.5)).  The paper
selects keyframes whose co-visibility exceeds 70% and a random 30% of the others.

Every step is a float32 operation in the order written below (numpy float32
arithmetic rounds each operation once), so the inside / outside decision of a
point has one answer; a float64 evaluation differs from it only for points within
rounding distance of an image border.
"""
from __future__ import annotations

import numpy as np

f32 = np.float32


def _pose(cam):
    m = np.asarray(cam["world_to_cam"], np.float32).reshape(3, 4)
    return m[:, :3], m[:, 3]


def observed_points(depth: np.ndarray, cam: dict, step: int) -> np.ndarray:
    """World points [n][3] float32 of the sampled pixels with depth > 0."""
    depth = np.asarray(depth, np.float32)
    H, W = depth.shape
    ys, xs = np.mgrid[0:H:step, 0:W:step]
    d = depth[ys, xs]
    keep = d > 0
    x, y, d = xs[keep].astype(np.float32), ys[keep].astype(np.float32), d[keep]
    xn = (x - f32(cam["cx"])) / f32(cam["fx"])
    yn = (y - f32(cam["cy"])) / f32(cam["fy"])
    R, t = _pose(cam)
    q = [xn * d - t[0], yn * d - t[1], d - t[2]]
    # R^T q, each component ((R0i q0 + R1i q1) + R2i q2)
    pw = [(R[0, i] * q[0] + R[1, i] * q[1]) + R[2, i] * q[2] for i in range(3)]
    return np.stack(pw, 1).astype(np.float32)


def inside(points: np.ndarray, cam: dict) -> np.ndarray:
    """Which world points [n][3] lie in front of cam and project into its image."""
    R, t = _pose(cam)
    p = np.asarray(points, np.float32)
    q = [((R[j, 0] * p[:, 0] + R[j, 1] * p[:, 1]) + R[j, 2] * p[:, 2]) + t[j] for j in range(3)]
    front = q[2] > f32(cam["znear"])
    with np.errstate(divide="ignore", invalid="ignore"):
        u = f32(cam["fx"]) * (q[0] / q[2]) + f32(cam["cx"])
        v = f32(cam["fy"]) * (q[1] / q[2]) + f32(cam["cy"])
    umax, vmax = f32(cam["width"]) - f32(0.5), f32(cam["height"]) - f32(0.5)
    return front & (u >= f32(-0.5)) & (u < umax) & (v >= f32(-0.5)) & (v < vmax)


def covisibility(depth: np.ndarray, cam: dict, keyframes: list, step: int):
    """(points inside each keyframe [K] int64, sampled points with depth > 0)."""
    pts = observed_points(depth, cam, step)
    return np.array([int(inside(pts, k).sum()) for k in keyframes], np.int64), int(pts.shape[0])


def select(inside_counts: np.ndarray, valid: int, u: np.ndarray, threshold: float = 0.7, frac: float = 0.3):
    """Kind per keyframe: 1 co-visible (inside / valid > threshold), 2 random (the
    round(frac * rest) non-co-visible keyframes with the smallest draws u, ties by
    index), 0 not selected."""
    n = len(inside_counts)
    thr = float(np.float32(threshold))
    covis = np.array([valid > 0 and float(c) > thr * float(valid) for c in inside_counts], bool)
    rest = np.flatnonzero(~covis)
    want = int(np.floor(f32(frac) * f32(len(rest)) + f32(0.5)))
    order = sorted(rest, key=lambda j: (np.float32(u[j]), j))
    kind = np.where(covis, 1, 0).astype(np.int32)
    kind[np.asarray(order[:want], np.int64)] = 2
    return kind
