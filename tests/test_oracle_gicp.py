"""Pins of the GICP tracking oracle (Sec. III-B, eq12-eq14): back-projection of a
fronto-parallel frame in closed form, voxel downsampling of a lattice, the plane
covariance of points on a known plane, the float32 neighbour selection against
brute force, and the recovery of a known rigid motion."""
import math

import numpy as np

from oracle import gicp as og
from paper_2503_01109_gb300 import synthetic as syn


def test_depth_points_closed_form_and_mask():
    cam = syn.pinhole(64, 48, 60.0)
    depth = np.full((48, 64), 2.5, np.float32)
    depth[10, 8] = 0.0                      # not a sampled pixel (y % 4 != 0)
    pts = og.depth_points(depth, cam, step=4)
    assert pts.shape == (16 * 12, 3)
    ys, xs = np.mgrid[0:48:4, 0:64:4]
    ref = np.stack([(xs - 31.5) / 60.0 * 2.5, (ys - 23.5) / 60.0 * 2.5, np.full(xs.shape, 2.5)], -1).reshape(-1, 3)
    assert np.allclose(pts, ref, rtol=0, atol=1e-6)
    depth[8, 8] = 0.0                       # a sampled pixel without depth is dropped
    assert og.depth_points(depth, cam, 4).shape[0] == 16 * 12 - 1
    mask = np.zeros((48, 64), np.uint8)
    mask[:, :32] = 4
    assert og.depth_points(depth, cam, 4, mask, 4).shape[0] == 8 * 12 - 1
    assert og.depth_points(depth, cam, 4, mask, 2).shape[0] == 0


def test_voxel_downsample_lattice():
    # a 0.25-cell lattice: 4^3 points in each cell of a 3x2x2-cell block, one kept per cell
    g = np.stack(np.meshgrid(np.arange(12), np.arange(8), np.arange(8), indexing="ij"), -1).reshape(-1, 3)
    pts = ((g + 0.5) * 0.025).astype(np.float32)
    pts = pts[np.random.default_rng(0).permutation(len(pts))]
    out = og.voxel_downsample(pts, (0, 0, 0), 0.1, (3, 2, 2))
    assert out.shape == (12, 3)
    c = og.cells(pts, (0, 0, 0), 0.1, (3, 2, 2))
    first = {int(ci): i for i, ci in reversed(list(enumerate(c)))}
    assert np.array_equal(out, pts[sorted(first.values())])
    out2 = og.voxel_downsample(np.vstack([pts, [[5.0, 5.0, 5.0]]]).astype(np.float32), (0, 0, 0), 0.1, (3, 2, 2))
    assert out2.shape == (12, 3)            # a point outside the grid is dropped


def test_plane_covariance_and_isolated_points():
    xs, ys = np.meshgrid(np.linspace(0, 1, 30), np.linspace(0, 1, 30))
    z = 0.3 * xs + 0.2 * ys + 1.0
    pts = np.stack([xs, ys, z], -1).reshape(-1, 3).astype(np.float32)
    pts = np.vstack([pts, [[5.0, 5.0, 5.0]]]).astype(np.float32)
    C = og.covariances(pts, 0.1, 10, 1e-3)
    n = np.array([-0.3, -0.2, 1.0]) / math.sqrt(0.09 + 0.04 + 1.0)
    ref = np.eye(3) - (1 - 1e-3) * np.outer(n, n)
    assert np.abs(C[:-1] - ref).max() < 2e-4     # float32 inputs: the plane is exact to ~1e-7
    assert np.array_equal(C[-1], np.eye(3))      # no neighbours: identity


def test_neighbour_selection_is_brute_force():
    rng = np.random.default_rng(1)
    pts = rng.uniform(0, 0.5, (400, 3)).astype(np.float32)
    nb = og.neighbours(pts, 0.08, 7)
    r2 = np.float32(0.08) * np.float32(0.08)
    for i in range(0, 400, 13):
        d2 = og.dist2_f32(pts[i][None], pts)
        js = np.flatnonzero(d2 <= r2)
        ref = js[np.lexsort((js, d2[js]))][:7]
        assert np.array_equal(nb[i], ref)
        assert nb[i][0] == i


def _corner(n=3000, seed=0):
    rng = np.random.default_rng(seed)
    u = rng.uniform(0, 1.5, (n, 2))
    face = rng.integers(0, 3, n)
    p = np.zeros((n, 3))
    for f in range(3):
        s = face == f
        others = [a for a in range(3) if a != f]
        p[s, others[0]], p[s, others[1]] = u[s, 0], u[s, 1]
    return p.astype(np.float32)


def test_gicp_recovers_a_known_motion():
    tgt = _corner()
    C = og.covariances(tgt, 0.15, 10, 1e-3)
    T_true = np.hstack([og.rodrigues([0.02, -0.03, 0.015]), [[0.03], [-0.02], [0.04]]])
    # the source sees the target from the moved frame: T_true maps it onto the target
    src = ((tgt.astype(np.float64) - T_true[:, 3]) @ T_true[:, :3]).astype(np.float32)
    Cs = og.covariances(src, 0.15, 10, 1e-3)
    T, stats = og.gicp(src, Cs, tgt, C, np.hstack([np.eye(3), np.zeros((3, 1))]), 30, 0.15, 0.05)
    # float32 source coordinates limit the match to ~1e-7
    assert np.abs(T[:, :3] - T_true[:, :3]).max() < 1e-5 and np.abs(T[:, 3] - T_true[:, 3]).max() < 1e-5
    assert stats[2] > 0.99 and stats[1] > 0.99 * len(src)
    _, s2 = og.gicp(src, Cs, tgt, C, T_true, 1, 0.15, 0.05)   # from the answer, the cost is at the noise floor
    assert s2[0] < 1e-6
