"""Oracle of the GICP tracking of Sec. III-B (eq12-eq14) on a sparse point map
(test infrastructure only).

Steps, in the paper's order and notation:

1. the observed points of a depth frame (pixels sampled every `step` px, depth
   > 0, optionally a mask), back-projected in camera coordinates;
2. uniform downsampling in 3D for the sparse map: one point per occupied cell of
   a grid (the lowest index), in index order;
3. the local-surface covariances C_p, C_q of eq12/eq13: for each point the (up
   to) k nearest points within a radius (itself included), their sample
   covariance, regularised to a plane: eps v1 v1^T + v2 v2^T + v3 v3^T with v1 the
   eigenvector of the smallest eigenvalue (identity with fewer than 3 points);
4. eq14 by Gauss-Newton: d_i = q_i - T p_i (eq12) with q_i the nearest target
   point to T p_i within max_dist; d_i ~ N(0, C_q + R C_p R^T) (eq13); the
   increment xi = (w, v) of T <- (Rodrigues(w), v) T solves the normal equations
   of the linearisation d + [[T p]_x, -I] xi; correspondences are renewed every
   iteration; it stops when |xi| < 1e-6, or keeps the pose when fewer than 6
   pairs or a singular system remain.

Steps 1 and 2 and the neighbour sets of step 3 are integer decisions taken on
float32 values; they are computed in float32 in the same operation order as the
kernels (each numpy float32 operation rounds once), so they agree exactly.  The
covariances and the Gauss-Newton iterations are FP64.  scipy's cKDTree supplies
candidate neighbours (a library search; the selection is decided here).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial import cKDTree

f32 = np.float32


def depth_points(depth: np.ndarray, cam: dict, step: int, mask: np.ndarray | None = None, bits: int = 0xFF):
    """Camera-frame points [n][3] float32 in pixel order."""
    depth = np.asarray(depth, np.float32)
    H, W = depth.shape
    ys, xs = np.mgrid[0:H:step, 0:W:step]
    d = depth[ys, xs]
    keep = d > 0
    if mask is not None:
        keep &= (np.asarray(mask)[ys, xs] & bits) != 0
    x, y, d = xs[keep].astype(np.float32), ys[keep].astype(np.float32), d[keep]
    px = ((x - f32(cam["cx"])) / f32(cam["fx"])) * d
    py = ((y - f32(cam["cy"])) / f32(cam["fy"])) * d
    return np.stack([px, py, d], 1).astype(np.float32)


def cells(points: np.ndarray, origin, cell: float, dims):
    """Cell index per point (-1 outside), decided in float32."""
    p = np.asarray(points, np.float32)
    c = np.floor((p - np.asarray(origin, np.float32)) / f32(cell)).astype(np.int64)
    inside = np.all((c >= 0) & (c < np.asarray(dims)), axis=1)
    idx = (c[:, 2] * dims[1] + c[:, 1]) * dims[0] + c[:, 0]
    return np.where(inside, idx, -1)


def voxel_downsample(points: np.ndarray, origin, cell: float, dims) -> np.ndarray:
    """The lowest-index point of every occupied cell, in index order."""
    c = cells(points, origin, cell, dims)
    seen, keep = set(), []
    for i, ci in enumerate(c.tolist()):
        if ci >= 0 and ci not in seen:
            seen.add(ci)
            keep.append(i)
    return np.asarray(points, np.float32)[np.asarray(keep, np.int64)]


def dist2_f32(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """((dx^2 + dy^2) + dz^2) in float32, the kernels' order."""
    d = np.asarray(a, np.float32) - np.asarray(b, np.float32)
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def neighbours(points: np.ndarray, radius: float, k: int, origin=None, dims=None):
    """Per point the (up to) k nearest points with float32 squared distance <= radius^2
    (itself included), ordered by (squared distance, index).  With a grid (origin,
    dims), points outside it have no neighbours and only points in the grid count."""
    p = np.asarray(points, np.float32)
    ok = np.ones(len(p), bool) if origin is None else cells(p, origin, radius, dims) >= 0
    tree = cKDTree(p.astype(np.float64))
    cand = tree.query_ball_point(p.astype(np.float64), r=float(radius) * 1.001 + 1e-7)
    r2 = f32(radius) * f32(radius)
    out = []
    for i, js in enumerate(cand):
        if not ok[i]:
            out.append(np.zeros(0, np.int64))
            continue
        js = np.asarray([j for j in js if ok[j]], np.int64)
        d2 = dist2_f32(p[i][None], p[js])
        sel = d2 <= r2
        js, d2 = js[sel], d2[sel]
        order = np.lexsort((js, d2))
        out.append(js[order][:k])
    return out


def covariances(points: np.ndarray, radius: float, k: int, eps: float, origin=None, dims=None) -> np.ndarray:
    """Regularised GICP covariances [n][3][3] (FP64)."""
    p = np.asarray(points, np.float64)
    nb = neighbours(points, radius, k, origin, dims)
    C = np.tile(np.eye(3), (len(p), 1, 1))
    for i, js in enumerate(nb):
        if len(js) < 3:
            continue
        q = p[js]
        dq = q - q.mean(0)
        S = dq.T @ dq / len(js)
        w, V = np.linalg.eigh(S)
        v1 = V[:, 0]
        C[i] = np.eye(3) - (1.0 - eps) * np.outer(v1, v1)
    return C


def eigen_gap(points: np.ndarray, radius: float, k: int, origin=None, dims=None) -> np.ndarray:
    """(lambda2 - lambda1) / lambda3 of each point's neighbourhood covariance (0 with
    fewer than 3 neighbours): where it is small the plane normal is ill-defined."""
    p = np.asarray(points, np.float64)
    out = np.zeros(len(p))
    for i, js in enumerate(neighbours(points, radius, k, origin, dims)):
        if len(js) < 3:
            continue
        dq = p[js] - p[js].mean(0)
        w = np.linalg.eigvalsh(dq.T @ dq / len(js))
        out[i] = (w[1] - w[0]) / max(w[2], 1e-300)
    return out


def skew(p):
    return np.array([[0.0, -p[2], p[1]], [p[2], 0.0, -p[0]], [-p[1], p[0], 0.0]])


def rodrigues(w):
    th = float(np.linalg.norm(w))
    if th < 1e-12:
        return np.eye(3) + skew(w)
    K = skew(np.asarray(w, np.float64) / th)
    return np.eye(3) + math.sin(th) * K + (1.0 - math.cos(th)) * (K @ K)


def gicp(src, src_cov, tgt, tgt_cov, pose0, iterations: int, max_dist: float, overlap_dist: float):
    """eq14 by Gauss-Newton.  pose0 [3][4] world-from-source.  Returns (pose [3][4],
    stats: cost and pairs at the last evaluated pose, overlap fraction there,
    iterations)."""
    src = np.asarray(src, np.float64)
    tgt = np.asarray(tgt, np.float64)
    Cp = np.asarray(src_cov, np.float64)
    Cq = np.asarray(tgt_cov, np.float64)
    T = np.asarray(pose0, np.float64).reshape(3, 4).copy()
    tree = cKDTree(tgt)
    stats = [0.0, 0.0, 0.0, 0.0]
    for it in range(iterations):
        R, t = T[:, :3], T[:, 3]
        P = src @ R.T + t
        dist, j = tree.query(P, k=1)
        stats[2] = float(np.mean(dist <= overlap_dist)) if len(P) else 0.0
        H = np.zeros((6, 6))
        b = np.zeros(6)
        cost, pairs = 0.0, 0
        for i in np.flatnonzero(dist <= max_dist):
            d = tgt[j[i]] - P[i]
            M = np.linalg.inv(Cq[j[i]] + R @ Cp[i] @ R.T)
            J = np.hstack([skew(P[i]), -np.eye(3)])
            H += J.T @ M @ J
            b += J.T @ M @ d
            cost += d @ M @ d
            pairs += 1
        stats[0], stats[1], stats[3] = cost, float(pairs), float(it + 1)
        if pairs < 6:
            break
        try:
            np.linalg.cholesky(H)
        except np.linalg.LinAlgError:
            break
        xi = -np.linalg.solve(H, b)
        Rw = rodrigues(xi[:3])
        T = np.hstack([Rw @ R, (Rw @ t + xi[3:])[:, None]])
        if np.linalg.norm(xi) < 1e-6:
            break
    return T, stats
