"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module draws inputs only: Gaussian parameters, cameras, trajectories and
random upstream gradients.  It holds none of the mapping method's arithmetic
(no projection, blending, filtering or seeding) and imports neither the CUDA
library nor the oracle.  The paper's datasets (Replica, TUM RGB-D) are not
available, so these scenes stand in for their shapes and sizes:

* ``tiny_scene``  -- 2,000 Gaussians in front of a 64x48 camera.
* ``room_scene``  -- Gaussians on the inner faces of a 4 x 3 x 3 m box, either a
  map to optimise (random colours, small isotropic-ish scales) or a ground-truth
  scene of flat and textured patches whose render is the optimisation target.
* ``room_camera`` / ``trajectory`` -- poses inside that room.

Every array is float32 in structure-of-arrays planes:
means[3][n], log_scales[3][n], quats[4][n] (w, x, y, z), logits[n], rgb[3][n].
World axes follow the camera convention at yaw = pitch = 0: x right, y down,
z forward.
"""
from __future__ import annotations

import math

import numpy as np

ROOM_HALF = np.array([2.0, 1.5, 1.5])  # 4 x 3 x 3 m box centred at the origin


def pinhole(width: int, height: int, f: float, world_to_cam=None, cx=None, cy=None,
            znear: float = 0.2) -> dict:
    """Pinhole camera dict; principal point at the image centre ((W-1)/2, (H-1)/2)."""
    if world_to_cam is None:
        world_to_cam = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    return {"width": int(width), "height": int(height), "fx": float(f), "fy": float(f),
            "cx": float((width - 1) / 2 if cx is None else cx), "cy": float((height - 1) / 2 if cy is None else cy),
            "world_to_cam": np.asarray(world_to_cam, np.float32).reshape(3, 4), "znear": float(znear)}


def _random_quats(rng, n):
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return q


def tiny_scene(n: int = 2000, seed: int = 0) -> dict:
    """Means uniform in [-1,1]^2 x [2,4], log-scales N(-3, 0.3), unit quaternions,
    opacity logits N(0, 1), RGB uniform in [0, 1] (SH degree 0)."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 4, n)])
    return _pack(means, rng.normal(-3.0, 0.3, (3, n)), _random_quats(rng, n), rng.normal(0.0, 1.0, n),
                 rng.uniform(0, 1, (3, n)))


EDGE_KINDS = ("clamp", "saturate", "near", "needle", "opaque")


def edge_scene(kind: str, n: int = 1500, seed: int = 0) -> dict:
    """Scenes for a 64x48 (or 70x45) camera with f = 60 at the identity pose that
    exercise the rare branches of projection and blending, each mixed with a
    tiny-scene background (means in [-1,1]^2 x [2,4]):

    * "clamp":    a third of the Gaussians beyond the Jacobian clamp in x
                  (|x/z| in [0.8, 1.1]), a third beyond it in y (|y/z| in
                  [0.58, 0.85]), large enough (log-scales N(-1, 0.3)) that their
                  footprints reach into the image;
    * "saturate": opacity logits N(5.5, 1), so o * G exceeds the 0.99 alpha clamp
                  near the centres;
    * "near":     half the means at depths in [0.1, 0.45] around the 0.2 near
                  plane (none within 1e-3 of it), small log-scales N(-5, 0.5);
    * "needle":   half the Gaussians needle-like (log-scales -1.5, -6.5, -6.5 in a
                  random axis order, random rotation): nearly degenerate 2D
                  covariances before the dilation;
    * "opaque":   a quarter large opaque Gaussians (log-scales N(-1.6, 0.2),
                  logits N(4, 0.5)), so that many pixels stop early (T < 1e-4)."""
    rng = np.random.default_rng(seed)
    base = tiny_scene(n, seed + 1000)
    means, ls, q = base["means"].astype(np.float64), base["log_scales"].astype(np.float64), base["quats"]
    logits, rgb = base["logits"].astype(np.float64), base["rgb"]
    if kind == "clamp":
        k = n // 3
        z = rng.uniform(2.0, 4.0, 2 * k)
        side = rng.choice([-1.0, 1.0], (2, 2 * k))
        u = rng.uniform(-0.5, 0.5, 2 * k)
        v = rng.uniform(-0.35, 0.35, 2 * k)
        u[:k] = side[0, :k] * rng.uniform(0.8, 1.1, k)           # beyond the x clamp
        v[k:] = side[1, k:] * rng.uniform(0.58, 0.85, k)         # beyond the y clamp
        both = rng.uniform(0, 1, 2 * k) < 0.2                    # some beyond both
        v[:k][both[:k]] = side[1, :k][both[:k]] * rng.uniform(0.58, 0.85, both[:k].sum())
        means[:, :2 * k] = np.stack([u * z, v * z, z])
        ls[:, :2 * k] = rng.normal(-1.0, 0.3, (3, 2 * k))
    elif kind == "saturate":
        logits = rng.normal(5.5, 1.0, n)
        ls = rng.normal(-2.6, 0.3, (3, n))
    elif kind == "near":
        k = n // 2
        z = rng.uniform(0.1, 0.45, k)
        z = np.where(np.abs(z - 0.2) < 1e-3, z + 2e-3, z)
        means[:, :k] = np.stack([rng.uniform(-0.4, 0.4, k) * z, rng.uniform(-0.3, 0.3, k) * z, z])
        ls[:, :k] = rng.normal(-5.0, 0.5, (3, k))
    elif kind == "needle":
        k = n // 2
        axis = rng.integers(0, 3, k)
        ls[:, :k] = -6.5
        ls[axis, np.arange(k)] = -1.5
    elif kind == "opaque":
        k = n // 4
        ls[:, :k] = rng.normal(-1.6, 0.2, (3, k))
        logits[:k] = rng.normal(4.0, 0.5, k)
    else:
        raise ValueError(kind)
    return _pack(means, ls, q, logits, rgb)


def _pack(means, log_scales, quats, logits, rgb) -> dict:
    return {"means": np.ascontiguousarray(means, np.float32),
            "log_scales": np.ascontiguousarray(log_scales, np.float32),
            "quats": np.ascontiguousarray(quats, np.float32),
            "logits": np.ascontiguousarray(logits, np.float32),
            "rgb": np.ascontiguousarray(rgb, np.float32)}


def _room_points(rng, n, jitter=0.01):
    """Uniform points on the six inner faces (area-weighted), jittered along the normal."""
    h = ROOM_HALF
    areas = np.array([4 * h[1] * h[2]] * 2 + [4 * h[0] * h[2]] * 2 + [4 * h[0] * h[1]] * 2)
    face = rng.choice(6, size=n, p=areas / areas.sum())
    u = rng.uniform(-1, 1, (2, n))
    p = np.zeros((3, n))
    normal_axis = face // 2
    sign = np.where(face % 2 == 0, -1.0, 1.0)
    for ax in range(3):
        sel = normal_axis == ax
        others = [a for a in range(3) if a != ax]
        p[ax, sel] = sign[sel] * h[ax] - sign[sel] * rng.uniform(-jitter, jitter, sel.sum())
        p[others[0], sel] = u[0, sel] * h[others[0]]
        p[others[1], sel] = u[1, sel] * h[others[1]]
    return p, face


def room_scene(n: int, seed: int, kind: str = "map") -> dict:
    """Gaussians on the room's inner faces (+-1 cm normal jitter).

    kind="map": parameters as the tiny scene (log-scales N(-3, 0.3), logits N(0, 1),
    RGB uniform).  kind="gt": half the area in flat patches (one colour per 0.5 m
    patch, log-scales N(-2.5, 0.3)), half textured (stripes or checkers of 7-27 mm
    period, i.e. 2-8 px at 2 m and f = 600, log-scales N(-3.5, 0.3)); opacity
    logits N(3, 0.5) so that the rendered depth is valid almost everywhere."""
    rng = np.random.default_rng(seed)
    p, face = _room_points(rng, n)
    q = _random_quats(rng, n)
    if kind == "map":
        return _pack(p, rng.normal(-3.0, 0.3, (3, n)), q, rng.normal(0.0, 1.0, n), rng.uniform(0, 1, (3, n)))
    if kind != "gt":
        raise ValueError(kind)
    # patch id from a 0.5 m grid on the face
    cell = np.floor((p + ROOM_HALF[:, None]) / 0.5).astype(np.int64)
    pid = face * 1_000_000 + cell[0] * 10_000 + cell[1] * 100 + cell[2]
    uniq, inv = np.unique(pid, return_inverse=True)
    prng = np.random.default_rng(seed + 7919)
    textured_patch = prng.uniform(0, 1, uniq.size) < 0.5
    base = prng.uniform(0.05, 0.95, (3, uniq.size))
    alt = prng.uniform(0.05, 0.95, (3, uniq.size))
    period = prng.uniform(0.007, 0.027, uniq.size)
    angle = prng.uniform(0, math.pi, uniq.size)
    checker = prng.uniform(0, 1, uniq.size) < 0.5
    tex = textured_patch[inv]
    # in-face coordinates: the two axes other than the face normal
    ax = face // 2
    a0 = np.where(ax == 0, p[1], p[0])
    a1 = np.where(ax == 2, p[1], p[2])
    c, s = np.cos(angle[inv]), np.sin(angle[inv])
    t0 = (c * a0 + s * a1) / period[inv]
    t1 = (-s * a0 + c * a1) / period[inv]
    stripe = (np.floor(t0) % 2 == 0)
    check = ((np.floor(t0) + np.floor(t1)) % 2 == 0)
    use_alt = np.where(checker[inv], check, stripe) & tex
    rgb = np.where(use_alt[None, :], alt[:, inv], base[:, inv])
    ls = np.where(tex[None, :], rng.normal(-3.5, 0.3, (3, n)), rng.normal(-2.5, 0.3, (3, n)))
    return _pack(p, ls, q, rng.normal(3.0, 0.5, n), rgb)


def look_pose(position, yaw: float, pitch: float = 0.0) -> np.ndarray:
    """world_to_cam [R | t] of a camera at `position` looking along (yaw, pitch)."""
    fwd = np.array([math.sin(yaw) * math.cos(pitch), -math.sin(pitch), math.cos(yaw) * math.cos(pitch)])
    down = np.array([0.0, 1.0, 0.0])
    right = np.cross(down, fwd)
    right /= np.linalg.norm(right)
    cam_down = np.cross(fwd, right)
    R = np.stack([right, cam_down, fwd])
    t = -R @ np.asarray(position, np.float64)
    return np.concatenate([R, t[:, None]], axis=1).astype(np.float32)


def room_camera(width: int, height: int, f: float, seed: int) -> dict:
    """A camera at a seeded position inside the room looking roughly horizontally."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1, 1, 3) * np.array([1.0, 0.5, 0.75])
    return pinhole(width, height, f, look_pose(pos, rng.uniform(-math.pi, math.pi), rng.uniform(-0.2, 0.2)))


def trajectory(n_frames: int, seed: int, width: int, height: int, f: float) -> list:
    """Smooth seeded trajectory: the sum of three low-frequency sinusoids on the
    position and a +-30 degree yaw sweep."""
    rng = np.random.default_rng(seed)
    p0 = rng.uniform(-0.3, 0.3, 3)
    amp = rng.uniform(0.05, 0.25, (3, 3)) * np.array([1.0, 0.4, 0.8])
    omega = rng.uniform(0.05, 0.2, 3)
    phase = rng.uniform(0, 2 * math.pi, (3, 3))
    yaw0 = rng.uniform(-math.pi, math.pi)
    cams = []
    for k in range(n_frames):
        pos = p0 + sum(amp[j] * np.sin(omega[j] * k + phase[j]) for j in range(3))
        yaw = yaw0 + math.radians(30) * math.sin(0.15 * k + phase[0, 0])
        cams.append(pinhole(width, height, f, look_pose(pos, yaw, 0.1 * math.sin(0.1 * k))))
    return cams


def random_image_grads(views: list, seed: int, scale: float = 1e-3) -> dict:
    """Seeded upstream gradients dL/dC [3][H][W], dL/dD and dL/dA per view,
    concatenated view after view."""
    rng = np.random.default_rng(seed)
    dC, dD, dA = [], [], []
    for cam in views:
        H, W = cam["height"], cam["width"]
        dC.append(rng.standard_normal((3, H, W)) * scale)
        dD.append(rng.standard_normal((H, W)) * scale)
        dA.append(rng.standard_normal((H, W)) * scale)
    return {"dC": [a.astype(np.float32) for a in dC], "dD": [a.astype(np.float32) for a in dD],
            "dA": [a.astype(np.float32) for a in dA]}


def subset(scene: dict, idx) -> dict:
    """Gaussians idx of a scene."""
    return {k: np.ascontiguousarray(v[..., idx]) for k, v in scene.items()}


def concat(a: dict, b: dict) -> dict:
    return {k: np.ascontiguousarray(np.concatenate([a[k], b[k]], axis=-1)) for k in a}


def textured_frame(width: int, height: int, seed: int) -> dict:
    """An RGB-D frame drawn directly (not rendered): flat patches and striped or
    checkered patches of 2-8 px period on a 16-px grid, plus a smooth depth map in
    [1.5, 4] m with a few invalid (0) pixels.  Returns rgb [3][H][W], depth [H][W]."""
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    rgb = np.zeros((3, height, width))
    cell = 16
    for cy in range(0, height, cell):
        for cx in range(0, width, cell):
            sl = (slice(cy, cy + cell), slice(cx, cx + cell))
            base = rng.uniform(0.1, 0.9, 3)
            if rng.uniform() < 0.5:
                alt = rng.uniform(0.1, 0.9, 3)
                period = rng.uniform(2, 8)
                ang = rng.uniform(0, math.pi)
                t = (np.cos(ang) * xs[sl] + np.sin(ang) * ys[sl]) / period
                on = (np.floor(t) % 2 == 0)
                for c in range(3):
                    rgb[c][sl] = np.where(on, alt[c], base[c])
            else:
                for c in range(3):
                    rgb[c][sl] = base[c]
    a, b, c0 = rng.uniform(-0.5, 0.5, 3)
    depth = 2.5 + a * (xs / width - 0.5) + b * (ys / height - 0.5) + 0.3 * np.sin(xs / 37.0 + c0) * np.cos(ys / 23.0)
    depth[rng.uniform(0, 1, depth.shape) < 0.01] = 0.0
    return {"rgb": rgb.astype(np.float32), "depth": depth.astype(np.float32)}


def fake_render(width: int, height: int, seed: int) -> dict:
    """Stand-in render outputs for the missing-region check: colour, unnormalised
    depth and opacity drawn at random (opacity spread around the 0.5 threshold)."""
    rng = np.random.default_rng(seed)
    A = np.clip(rng.uniform(-0.2, 1.2, (height, width)), 0.0, 1.0)
    D = rng.uniform(1.5, 4.0, (height, width)) * A
    C = rng.uniform(0, 1, (3, height, width))
    return {"color": C.astype(np.float32), "depth": D.astype(np.float32), "alpha": A.astype(np.float32)}


def box_depth(cam: dict, half=ROOM_HALF) -> np.ndarray:
    """Depth [H][W] (camera z) of the inside of an axis-aligned box centred at the
    origin, seen from a camera inside it: each pixel's ray hits the first face in
    its direction of travel.  An exact, view-consistent geometry for tracking."""
    W, H = cam["width"], cam["height"]
    M = np.asarray(cam["world_to_cam"], np.float64).reshape(3, 4)
    R, t = M[:, :3], M[:, 3]
    o = -R.T @ t
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    dc = np.stack([(xs - cam["cx"]) / cam["fx"], (ys - cam["cy"]) / cam["fy"], np.ones_like(xs)], -1)
    dw = dc @ R                                   # R^T d for every pixel
    h = np.asarray(half, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ts = np.where(dw > 0, (h - o) / dw, np.where(dw < 0, (-h - o) / dw, np.inf))
    return ts.min(-1).astype(np.float32)         # the ray parameter is the camera z (d_c.z = 1)


def corner_trajectory(n_frames: int, width: int, height: int, f: float, corner=(2.0, 1.5, 1.5)) -> list:
    """Cameras drifting slowly near the room centre while looking at a corner of the
    room, so that three faces are in view (every pose is then fixed by geometry)."""
    cams = []
    for k in range(n_frames):
        p = np.array([0.3 + 0.015 * k, 0.2 + 0.004 * k, 0.25 + 0.01 * math.sin(0.3 * k)])
        d = np.asarray(corner, np.float64) - p
        yaw = math.atan2(d[0], d[2]) + 0.01 * k
        pitch = -math.asin(d[1] / np.linalg.norm(d))
        cams.append(pinhole(width, height, f, look_pose(p, yaw, pitch)))
    return cams
