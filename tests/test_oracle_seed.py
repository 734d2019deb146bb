"""Pins of the Fourier-seeding oracle (Sec. III-A) against library routines,
closed forms and hand-built cases."""
import math
import os

import numpy as np
import pytest

from oracle import seed as osd
from paper_2503_01109_gb300 import synthetic as syn


def direct_dft2(I):
    """eq2 as the literal double sum (O((HW)^2)), for tiny images."""
    H, W = I.shape
    F = np.zeros((H, W), complex)
    for v in range(H):
        for u in range(W):
            acc = 0j
            for y in range(H):
                for x in range(W):
                    acc += I[y, x] * np.exp(-2j * math.pi * (u * x / W + v * y / H))
            F[v, u] = acc
    return F


def test_dft_equals_literal_sum_and_fft():
    rng = np.random.default_rng(0)
    I = rng.uniform(0, 1, (8, 8))
    F = osd.dft2(I)
    assert np.abs(F - direct_dft2(I)).max() < 1e-12
    for shape in [(8, 8), (48, 64), (17, 10)]:
        J = rng.uniform(0, 1, shape)
        assert np.abs(osd.dft2(J) - np.fft.fft2(J)).max() < 1e-9 * shape[0] * shape[1]
        assert np.abs(osd.idft2(osd.dft2(J)) - J).max() < 1e-12


def test_parseval_and_pure_cosine():
    H, W, k0 = 48, 64, 5
    x = np.arange(W)
    I = np.tile(np.cos(2 * math.pi * k0 * x / W), (H, 1))
    F = osd.dft2(I)
    assert abs(F[0, k0]) == pytest.approx(H * W / 2, rel=1e-12)
    assert abs(F[0, W - k0]) == pytest.approx(H * W / 2, rel=1e-12)
    mask = np.ones_like(F, bool); mask[0, k0] = mask[0, W - k0] = False
    assert np.abs(F[mask]).max() < 1e-9
    assert (np.abs(I) ** 2).sum() == pytest.approx((np.abs(F) ** 2).sum() / (H * W), rel=1e-12)


def test_centre_matches_fftshift():
    rng = np.random.default_rng(1)
    for shape in [(48, 64), (7, 9)]:
        F = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        assert np.array_equal(osd.centre(F), np.fft.fftshift(F))
        assert np.array_equal(osd.uncentre(osd.centre(F)), F)


def test_constant_frame_has_no_high_frequency_energy():
    """H(centre) = 0 removes the DC term: a constant frame has E = 0 everywhere."""
    rgb = np.full((3, 48, 64), 0.37)
    E = osd.high_frequency_energy(rgb, 0.25)
    assert E.max() < 1e-12
    assert osd.bins_f64(np.zeros((4, 4))).max() == 0
    # the rounding noise left in E is below the noise floor: no high-frequency bins
    assert osd.bins_f64(E, 0.37).max() == 0
    assert osd.bins_f32(E.astype(np.float32), np.float32(0.37)).max() == 0
    out = osd.seed_frame(rgb, np.ones((48, 64)), syn.pinhole(64, 48, 60.0))
    assert not (out["mask"] & 1).any() and not out["is_high"].any()


@pytest.mark.parametrize("k0,d0", [(5, 0.25), (20, 0.25), (3, 0.1)])
def test_highpass_of_cosine_closed_form(k0, d0):
    """I = cos(2 pi k0 x / W) gives I_h = H(k0) I with H(k0) = 1 - exp(-(k0/(W/2))^2 / (2 d0^2))."""
    H, W = 48, 64
    x = np.arange(W)
    g = np.tile(np.cos(2 * math.pi * k0 * x / W), (H, 1))
    rgb = np.stack([g, g, g])          # luma of a gray frame is the frame itself
    E = osd.high_frequency_energy(rgb, d0)
    h = 1 - math.exp(-((k0 / (W / 2)) ** 2) / (2 * d0 * d0))
    assert np.abs(E - np.abs(h * g)).max() < 1e-12


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            lhs, rhs = line.split("->")
            yield lhs.split(), rhs.strip()


def test_triangle_threshold_hand_built():
    cases = list(_golden_lines("triangle_threshold.txt"))
    assert len(cases) == 4
    for bins, t in cases:
        h = np.zeros(256, int)
        for b in bins:
            i, c = b.split(":")
            h[int(i)] = int(c)
        assert osd.triangle_threshold(h) == int(t), bins
    # far end ties resolve to the high side
    h = np.zeros(256, int); h[[3, 5, 7]] = [1, 9, 1]
    assert osd.triangle_threshold(h) in (5, 6, 7)


def test_bins_f32():
    E = np.array([0.0, 1.0, 0.5, 0.999999, 1e-9], np.float32)
    b = osd.bins_f32(E)
    assert list(b) == [0, 255, 128, 255, 0]


def test_missing_mask_hand_built():
    cases = [([float(x) for x in lhs], int(rhs)) for lhs, rhs in _golden_lines("missing_mask.txt")]
    assert len(cases) == 6
    v = np.array([c[0] for c in cases], np.float32)
    H, W = 1, len(cases)
    A, D, Dg = v[:, 0][None], v[:, 1][None], v[:, 2][None]
    C = np.zeros((3, H, W), np.float32)
    Cg = np.broadcast_to(v[:, 3][None, None], (3, H, W)).astype(np.float32)
    M = osd.missing_mask_f32(C, D, A, Cg, Dg)
    assert [int(x) for x in M[0]] == [c[1] for c in cases]


def test_seed_selection_order_grid_and_cap():
    H, W = 8, 16
    Mh = np.zeros((H, W), bool); Mh[:, :8] = True
    Mm = np.ones((H, W), bool); Mm[0, 0] = False
    depth = np.ones((H, W)); depth[2, 2] = 0
    xy, hi = osd.select_seeds(Mh, Mm, depth, m=2, n=8, max_new=1000)
    high = [(x, y) for x, y in xy[hi]]
    low = [(x, y) for x, y in xy[~hi]]
    expect_high = [(x, y) for y in range(0, H, 2) for x in range(0, 8, 2) if (x, y) not in [(0, 0), (2, 2)]]
    assert high == expect_high
    assert low == [(8, 0)]
    assert hi[: len(expect_high)].all() and not hi[len(expect_high):].any()
    xy2, _ = osd.select_seeds(Mh, Mm, depth, 2, 8, max_new=5)
    assert np.array_equal(xy2, xy[:5])


def test_backprojection_reprojects_and_eq11_scale():
    rng = np.random.default_rng(7)
    pose = syn.look_pose([0.2, 0.1, -0.3], 0.7, 0.05).astype(np.float64)
    cam = syn.pinhole(40, 30, 50.0, pose)
    cam["world_to_cam"] = pose
    depth = rng.uniform(0.5, 4.0, (30, 40))
    rgb = rng.uniform(0, 1, (3, 30, 40))
    xy = np.array([[0, 0], [39, 29], [17, 11], [5, 22]], np.int32)
    hi = np.array([True, False, True, False])
    g = osd.new_gaussians(xy, hi, rgb, depth, cam, alpha_h=1.0, alpha_l=4.0)
    R, t = pose[:, :3], pose[:, 3]
    pc = R @ g["means"] + t[:, None]
    u = 50.0 * pc[0] / pc[2] + cam["cx"]
    v = 50.0 * pc[1] / pc[2] + cam["cy"]
    assert np.abs(u - xy[:, 0]).max() < 1e-9 and np.abs(v - xy[:, 1]).max() < 1e-9
    d = depth[xy[:, 1], xy[:, 0]]
    assert g["log_scales"][0] == pytest.approx(np.log(np.where(hi, 1.0, 4.0) * d / 50.0), rel=1e-12)
    assert np.array_equal(g["quats"][:, 0], [1, 0, 0, 0])


def test_seed_frame_stripes_are_high_frequency():
    """Left half flat, right half 2-px stripes: the high-frequency mask covers the
    stripes and not the flat half away from the seams (the DFT is periodic, so
    column 0 borders the stripes too)."""
    H, W = 48, 64
    img = np.full((H, W), 0.5)
    img[:, 32:] = np.where((np.arange(32, W) // 2) % 2 == 0, 0.9, 0.1)[None, :]
    rgb = np.stack([img, img, img])
    out = osd.seed_frame(rgb, np.ones((H, W)), syn.pinhole(W, H, 60.0))
    Mh = (out["mask"] & 1).astype(bool)
    assert Mh[:, 40:60].mean() > 0.9
    assert Mh[:, 6:26].mean() < 0.05
    assert out["xy"].shape[0] > 0 and out["is_high"].any()
