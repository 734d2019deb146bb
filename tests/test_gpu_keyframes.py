"""Keyframe co-visibility and window selection on the GPU against the oracle:
counts and selections exact (the decisions are float32 on both sides)."""
import numpy as np
import pytest
import torch

from oracle import keyframes as ok
from paper_2503_01109_gb300 import fgs, synthetic as syn

pytestmark = pytest.mark.gpu


def _run(depth, cam, kfs, step):
    K = len(kfs)
    inside = torch.zeros(K, dtype=torch.int64, device="cuda")
    valid = torch.zeros(1, dtype=torch.int64, device="cuda")
    fgs.fgs_covisibility(torch.as_tensor(depth).cuda(), cam, kfs, step, inside, valid)
    return inside.cpu().numpy(), int(valid.item())


@pytest.mark.parametrize("W,H,step", [(1200, 680, 4), (640, 480, 1), (64, 48, 3)])
def test_covisibility_counts_match_oracle(cuda_device, W, H, step):
    f = 600.0 if W == 1200 else (525.0 if W == 640 else 60.0)
    cams = syn.trajectory(40, seed=100, width=W, height=H, f=f)
    depth = syn.textured_frame(W, H, seed=5)["depth"]
    cur = cams[20]
    kfs = cams[:20] + cams[21:] + [syn.room_camera(W, H, f, seed=s) for s in range(10)]
    got, valid = _run(depth, cur, kfs, step)
    ref, rvalid = ok.covisibility(depth, cur, kfs, step)
    assert valid == rvalid and np.array_equal(got, ref)
    assert got.max() > 0 and got.min() < valid          # some overlap, not all


def test_many_keyframes_and_selection(cuda_device):
    W, H, f = 640, 480, 525.0
    cams = syn.trajectory(200, seed=7, width=W, height=H, f=f)
    depth = syn.textured_frame(W, H, seed=6)["depth"]
    got, valid = _run(depth, cams[100], cams[:100] + cams[101:] + cams[:57], 2)   # 256 keyframes
    ref, _ = ok.covisibility(depth, cams[100], cams[:100] + cams[101:] + cams[:57], 2)
    assert np.array_equal(got, ref)
    u = np.random.default_rng(0).random(len(got)).astype(np.float32)
    kind = torch.zeros(len(got), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    fgs.fgs_select_keyframes(torch.as_tensor(got).cuda(), torch.tensor([valid], device="cuda"),
                             torch.as_tensor(u).cuda(), 0.7, 0.3, kind, count)
    want = ok.select(got, valid, u, 0.7, 0.3)
    assert np.array_equal(kind.cpu().numpy(), want) and int(count.item()) == int((want > 0).sum())
    assert (want == 1).any() and (want == 2).any()


def test_argument_errors(cuda_device):
    cam = syn.pinhole(32, 24, 30.0)
    d = torch.ones(24, 32, device="cuda")
    inside = torch.zeros(300, dtype=torch.int64, device="cuda")
    valid = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(fgs.FGSError):
        fgs.fgs_covisibility(d, cam, [cam] * 257, 1, inside, valid)
    with pytest.raises(fgs.FGSError):
        fgs.fgs_covisibility(d, cam, [cam], 0, inside, valid)
