"""GICP tracking on the GPU (Sec. III-B, eq12-eq14) against the oracle: the
observed points and the voxel downsampling bit-exact, the grid index complete,
the plane covariances and the Gauss-Newton pose within float32 reach of the FP64
oracle, and a synthetic trajectory tracked to a fraction of a millimetre."""
import numpy as np
import pytest
import torch

from oracle import gicp as og
from paper_2503_01109_gb300 import fgs, synthetic as syn
from paper_2503_01109_gb300.tracking import SparseMap, Tracker, cam_pose_inverse

pytestmark = pytest.mark.gpu

ROOM_GRID = ((-2.5, -2.0, -2.0), (50, 40, 40))   # the room box with a margin, 0.1 m cells
VOX = ((-2.5, -2.0, -2.0), (167, 134, 134))      # 0.03 m voxels over the same box


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def _n(k):
    return torch.tensor([int(k)], dtype=torch.int64, device="cuda")


def test_depth_points_bit_exact(cuda_device):
    cam = syn.room_camera(1200, 680, 600.0, seed=2)
    fr = syn.textured_frame(1200, 680, seed=3)
    mask = (np.arange(1200 * 680).reshape(680, 1200) % 7).astype(np.uint8)
    n = _n(0)
    for step, m, bits in ((8, None, 0xFF), (3, mask, 4)):
        cap = ((1200 + step - 1) // step) * ((680 + step - 1) // step)
        xyz = torch.zeros(cap, 3, device="cuda")
        ws = fgs.ws_tensor(fgs.fgs_depth_points_workspace_size(1200, 680, step))
        fgs.fgs_depth_points(_dev(fr["depth"]), None if m is None else _dev(m, torch.uint8), bits, cam, step, xyz, n,
                             ws)
        ref = og.depth_points(fr["depth"], cam, step, m, bits)
        k = int(n.item())
        assert k == len(ref) and np.array_equal(xyz[:k].cpu().numpy(), ref)
    # capacity overflow: truncated in order, status set
    xyz = torch.zeros(100, 3, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = fgs.ws_tensor(fgs.fgs_depth_points_workspace_size(1200, 680, 8))
    fgs.fgs_depth_points(_dev(fr["depth"]), None, 0xFF, cam, 8, xyz, n, ws, status)
    assert int(n.item()) == 100 and int(status.item()) & 8
    assert np.array_equal(xyz.cpu().numpy(), og.depth_points(fr["depth"], cam, 8)[:100])


def _room_points(n, seed):
    return np.ascontiguousarray(syn.room_scene(n, seed=seed, kind="map")["means"].T, np.float32)


def test_voxel_downsample_and_grid(cuda_device):
    pts = _room_points(200_000, 4)
    g = fgs.grid(ROOM_GRID[0], 0.05, (100, 80, 80))
    out = torch.zeros(len(pts), 3, device="cuda")
    n_out = _n(7)                                  # appended after 7 existing points
    ws = fgs.ws_tensor(fgs.fgs_voxel_workspace_size(g, len(pts)))
    fgs.fgs_voxel_downsample(_dev(pts), _n(len(pts)), g, ws, out, n_out)
    ref = og.voxel_downsample(pts, ROOM_GRID[0], 0.05, (100, 80, 80))
    k = int(n_out.item()) - 7
    assert k == len(ref) and np.array_equal(out[7:7 + k].cpu().numpy(), ref)
    # grid index of the downsampled cloud: every point once, in its own cell
    gg = fgs.grid(ROOM_GRID[0], 0.1, ROOM_GRID[1])
    cs = torch.zeros(fgs.grid_cells(gg) + 1, dtype=torch.int32, device="cuda")
    order = torch.zeros(len(ref), dtype=torch.int32, device="cuda")
    fgs.fgs_grid_build(_dev(ref), _n(len(ref)), gg, cs, order,
                       fgs.ws_tensor(fgs.fgs_grid_workspace_size(gg, len(ref))))
    cs, order = cs.cpu().numpy(), order.cpu().numpy()
    cells = og.cells(ref, ROOM_GRID[0], 0.1, ROOM_GRID[1])
    assert cs[-1] == int((cells >= 0).sum()) and np.all(np.diff(cs) >= 0)
    assert sorted(order[:cs[-1]].tolist()) == sorted(np.flatnonzero(cells >= 0).tolist())
    for c in np.unique(cells[cells >= 0])[::97]:
        assert set(order[cs[c]:cs[c + 1]].tolist()) == set(np.flatnonzero(cells == c).tolist())


def _cloud(pts, g, k=10, eps=1e-3):
    xyz, n = _dev(pts), _n(len(pts))
    cs = torch.zeros(fgs.grid_cells(g) + 1, dtype=torch.int32, device="cuda")
    order = torch.zeros(len(pts), dtype=torch.int32, device="cuda")
    fgs.fgs_grid_build(xyz, n, g, cs, order, fgs.ws_tensor(fgs.fgs_grid_workspace_size(g, len(pts))))
    cov = torch.zeros(len(pts), 6, device="cuda")
    fgs.fgs_point_covariances(xyz, n, g, cs, order, k, eps, cov)
    return xyz, n, cs, order, cov


def _full(c6):
    c = np.asarray(c6, np.float64)
    return np.stack([c[:, [0, 1, 2]], c[:, [1, 3, 4]], c[:, [2, 4, 5]]], 1)


def test_covariances_match_oracle(cuda_device):
    pts = og.voxel_downsample(_room_points(300_000, 5), VOX[0], 0.03, VOX[1])
    gg = fgs.grid(ROOM_GRID[0], 0.1, ROOM_GRID[1])
    *_, cov = _cloud(pts, gg)
    got = _full(cov.cpu().numpy())
    ref = og.covariances(pts, 0.1, 10, 1e-3, ROOM_GRID[0], ROOM_GRID[1])
    gap = og.eigen_gap(pts, 0.1, 10, ROOM_GRID[0], ROOM_GRID[1])
    clear = gap > 0.05
    assert clear.mean() > 0.9
    assert np.abs(got[clear] - ref[clear]).max() < 2e-3
    alone = gap == 0
    if alone.any():
        assert np.abs(got[alone] - np.eye(3)).max() == 0.0


def test_transform_points(cuda_device):
    pts = _room_points(10_000, 6)
    cov = np.tile(np.array([1.0, 0.1, 0.0, 2.0, 0.2, 3.0], np.float32), (len(pts), 1))
    T = np.hstack([og.rodrigues([0.3, -0.2, 0.1]), [[0.5], [-0.1], [0.2]]])
    xo, co = torch.zeros(len(pts), 3, device="cuda"), torch.zeros(len(pts), 6, device="cuda")
    fgs.fgs_transform_points(_dev(pts), _dev(cov), _n(len(pts)), _dev(T.reshape(-1), torch.float64), xo, co)
    assert np.abs(xo.cpu().numpy() - (pts @ T[:, :3].T + T[:, 3])).max() < 1e-5
    C = _full(cov[:1])[0]
    assert np.abs(_full(co.cpu().numpy()[:1])[0] - T[:, :3] @ C @ T[:, :3].T).max() < 1e-5


def test_gicp_matches_oracle(cuda_device):
    tgt = og.voxel_downsample(_room_points(400_000, 7), VOX[0], 0.03, VOX[1])
    gg = fgs.grid(ROOM_GRID[0], 0.1, ROOM_GRID[1])
    txyz, tn, cs, order, tcov = _cloud(tgt, gg)
    T_true = np.hstack([og.rodrigues([0.01, -0.015, 0.02]), [[0.03], [0.02], [-0.025]]])
    sel = np.random.default_rng(8).choice(len(tgt), 20_000, replace=False)
    src = ((tgt[sel].astype(np.float64) - T_true[:, 3]) @ T_true[:, :3]).astype(np.float32)
    sxyz, sn, _, _, scov = _cloud(src, fgs.grid((-3.0, -3.0, -3.0), 0.1, (60, 60, 60)))
    I = np.hstack([np.eye(3), np.zeros((3, 1))])
    pose = _dev(I.reshape(-1), torch.float64)
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    fgs.fgs_gicp(sxyz, scov, sn, txyz, tcov, gg, cs, order, fgs.GicpParams(25, 0.1, 0.05), pose, stats,
                 fgs.ws_tensor(fgs.fgs_gicp_workspace_size(len(src))))
    T = pose.cpu().numpy().reshape(3, 4)
    Tr, _ = og.gicp(src, _full(scov.cpu().numpy()), tgt, _full(tcov.cpu().numpy()), I, 25, 0.1, 0.05)
    assert np.abs(T - Tr).max() < 1e-4                     # float32 evaluation vs FP64
    assert np.abs(T - T_true).max() < 1e-4
    st = stats.cpu().numpy()
    assert st[2] > 0.99 and st[1] > 0.99 * len(src) and 1 <= st[3] <= 25


def test_gicp_argument_errors(cuda_device):
    g = fgs.grid((0, 0, 0), 0.1, (4, 4, 4))
    x = torch.zeros(8, 3, device="cuda")
    c = torch.zeros(8, 6, device="cuda")
    i = torch.zeros(65, dtype=torch.int32, device="cuda")
    pose, stats = torch.zeros(12, dtype=torch.float64, device="cuda"), torch.zeros(4, dtype=torch.float64, device="cuda")
    ws = fgs.ws_tensor(fgs.fgs_gicp_workspace_size(8))
    with pytest.raises(fgs.FGSError):   # correspondence distance beyond the grid's cell
        fgs.fgs_gicp(x, c, _n(8), x, c, g, i, i, fgs.GicpParams(5, 0.2, 0.05), pose, stats, ws)
    with pytest.raises(fgs.FGSError):
        fgs.fgs_gicp(x, c, _n(8), x, c, fgs.grid((0, 0, 0), 0.1, (1 << 10, 1 << 10, 1 << 10)), i, i,
                     fgs.GicpParams(5, 0.1, 0.05), pose, stats, ws)


def test_tracking_a_trajectory(cuda_device):
    # exact depth of the room box seen by cameras that look at a corner (three faces
    # in view fix all six degrees of freedom); the map grows by keyframes
    W, H, f = 640, 480, 525.0
    cams = syn.corner_trajectory(12, W, H, f)
    smap = SparseMap(fgs.grid(ROOM_GRID[0], 0.1, ROOM_GRID[1]), fgs.grid(VOX[0], 0.03, VOX[1]))
    tr = Tracker(cams[0], smap, fgs.grid((-6.0, -6.0, 0.0), 0.1, (120, 120, 80)), step=4)
    truth = [cam_pose_inverse(c["world_to_cam"]) for c in cams]
    tr.observe(_dev(syn.box_depth(cams[0])))
    tr.add_keyframe(truth[0])
    est, err, rot = truth[0], [], []
    for k in range(1, len(cams)):
        tr.observe(_dev(syn.box_depth(cams[k])))
        est, stats = tr.track(est)
        err.append(float(np.linalg.norm(est[:, 3] - truth[k][:, 3])))
        rot.append(float(np.abs(est[:, :3] - truth[k][:, :3]).max()))
        if stats[2] < 0.9:
            tr.add_keyframe(est)
    ate = float(np.sqrt(np.mean(np.square(err))))
    assert ate < 5e-4 and max(rot) < 5e-4, (ate, err, rot)
