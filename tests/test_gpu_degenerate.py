"""Degenerate and extreme inputs of the render path, through the C ABI: an empty
map, a map whose Gaussians are all behind the near plane, one Gaussian against
its closed-form footprint, the maximum number of views in one call, and
Gaussians so close to the camera that they cover every tile."""
import math

import numpy as np
import pytest
import torch

from oracle import render as orr
from paper_2503_01109_gb300 import fgs, synthetic as syn

from gpu_helpers import (PIX_TOL, assert_grads_exact, gpu_lists, gpu_view_splats, make_mapper, masked, oracle_flags,
                         tile_origin, to_device)

pytestmark = pytest.mark.gpu


def _background_only(m, cams):
    torch.cuda.synchronize()
    assert int(m.status.item()) == 0
    assert int(m.num_pairs.item()) == 0
    for v in range(len(cams)):
        out = m.frame.view(v)
        for key in ("color", "depth", "alpha"):
            assert torch.count_nonzero(out[key]).item() == 0, key
        assert torch.all(out["t_final"] == 1.0)
        assert torch.count_nonzero(out["n_contrib"]).item() == 0


def test_empty_map_renders_background_and_zero_gradients(cuda_device):
    cams = [syn.pinhole(70, 45, 60.0), syn.pinhole(33, 20, 30.0)]
    empty = {"means": np.zeros((3, 0), np.float32), "log_scales": np.zeros((3, 0), np.float32),
             "quats": np.zeros((4, 0), np.float32), "logits": np.zeros(0, np.float32),
             "rgb": np.zeros((3, 0), np.float32)}
    m = make_mapper(empty, cams, capacity=16)
    m.render()
    _background_only(m, cams)
    rg = syn.random_image_grads(cams, 1)
    m.backward(to_device(rg["dC"]), to_device(rg["dD"]), to_device(rg["dA"]))
    torch.cuda.synchronize()
    assert torch.count_nonzero(m.grads.buf).item() == 0


def test_every_gaussian_behind_the_near_plane(cuda_device):
    sc = syn.tiny_scene(500, seed=4)
    sc["means"][2] = np.random.default_rng(4).uniform(-3.0, 0.19, 500).astype(np.float32)
    cams = [syn.pinhole(64, 48, 60.0)]
    m = make_mapper(sc, cams)
    m.render()
    _background_only(m, cams)
    assert int((m.proj.radius[0, :500] > 0).sum().item()) == 0


def test_single_gaussian_closed_form(cuda_device):
    """One isotropic Gaussian on the optical axis at depth z with scale s and
    opacity o: alpha(x, y) = min(0.99, o exp(-r^2 / (2 ((f s / z)^2 + 0.3)))) inside
    its support, colour = c alpha, depth = z alpha (float32 within 2e-6)."""
    z, s, logit, rgb = 2.5, 0.04, 0.7, (0.2, 0.6, 0.9)
    sc = {"means": np.array([[0.0], [0.0], [z]], np.float32), "log_scales": np.full((3, 1), math.log(s), np.float32),
          "quats": np.array([[1.0], [0.0], [0.0], [0.0]], np.float32), "logits": np.array([logit], np.float32),
          "rgb": np.array(rgb, np.float32).reshape(3, 1)}
    cam = syn.pinhole(64, 48, 60.0)
    m = make_mapper(sc, [cam])
    m.render()
    torch.cuda.synchronize()
    out = m.frame.view(0)
    var = (60.0 * np.float32(s) / z) ** 2 + 0.3
    o = 1.0 / (1.0 + math.exp(-logit))
    ys, xs = np.mgrid[0:48, 0:64].astype(np.float64)
    a = np.minimum(0.99, o * np.exp(-((xs - 31.5) ** 2 + (ys - 23.5) ** 2) / (2 * var)))
    a[a < 1 / 255] = 0.0
    got = out["alpha"].cpu().numpy()
    support = got > 0
    # the support equals the closed form's (alpha >= 1/255, all inside the splat's tiles) except where the
    # closed-form alpha is within float32 reach of 1/255
    differ = support != (a > 0)
    assert not differ.any() or np.abs(np.minimum(0.99, o * np.exp(-((xs - 31.5) ** 2 + (ys - 23.5) ** 2) /
                                                                  (2 * var)))[differ] - 1 / 255).max() < 1e-8
    assert np.abs(got - a)[support].max() < 2e-6
    assert np.abs(out["depth"].cpu().numpy() - z * a)[support].max() < 2e-5
    for c in range(3):
        assert np.abs(out["color"].cpu().numpy()[c] - rgb[c] * a)[support].max() < 2e-6


def test_maximum_number_of_views(cuda_device):
    """FGS_MAX_VIEWS views of different sizes and poses in one call: lists bit-exact
    (teacher-forced) and every view's forward within 1e-4 outside the band."""
    rng = np.random.default_rng(3)
    cams = []
    for v in range(fgs.MAX_VIEWS):
        w, h = int(rng.integers(20, 60)), int(rng.integers(16, 40))
        pose = syn.look_pose(rng.uniform(-0.1, 0.1, 3), rng.uniform(-0.15, 0.15), rng.uniform(-0.1, 0.1))
        cams.append(syn.pinhole(w, h, 0.9 * w, pose))
    n = 800
    sc = syn.tiny_scene(n, seed=21)
    m = make_mapper(sc, cams)
    m.render()
    torch.cuda.synchronize()
    tk, ids, ranges = gpu_lists(m)
    V = len(cams)
    depth = np.stack([m.proj.splat[v, :n, 6].cpu().numpy() for v in range(V)]).astype(np.float32)
    radius = np.stack([m.proj.radius[v, :n].cpu().numpy() for v in range(V)])
    rect = np.stack([m.proj.rect[v, :n].cpu().numpy().view(np.uint16).astype(np.int32) for v in range(V)])
    supp = np.stack([orr.support_f32(m.proj.splat[v, :n].cpu().numpy()) for v in range(V)])
    rt, rids, rranges = orr.bin_sort(cams, 16, 16, depth, radius, rect, supp)
    assert np.array_equal(tk, rt) and np.array_equal(ids, rids) and np.array_equal(ranges, rranges)
    rgb = orr.aos(sc)["rgb"]
    bases = tile_origin(cams, 16, 16)
    for v, cam in enumerate(cams):
        gsp, _ = gpu_view_splats(m, v, n)
        ref = orr.render_fwd(gsp, rgb, cam, ids, ranges, bases[v], 16, 16)
        out = m.frame.view(v)
        ok = ref["flag"] == 0
        assert np.abs(out["color"].cpu().numpy() - ref["color"])[:, ok].max() <= PIX_TOL
        assert np.array_equal(out["n_contrib"].cpu().numpy()[ok], ref["n_contrib"][ok])
    with pytest.raises(fgs.FGSError):
        fgs.fgs_project(m.g, cams + cams[:1], m.til, m.proj)


def test_gaussians_covering_every_tile(cuda_device):
    """A few large Gaussians just beyond the near plane cover the whole image in
    front of an ordinary scene: every tile's list holds them; forward and every
    gradient entry match the oracle (band pixels masked)."""
    base = syn.tiny_scene(1200, seed=31)
    big = {"means": np.array([[0.0, 0.05, -0.04], [0.0, -0.03, 0.02], [0.3, 0.35, 0.45]], np.float32),
           "log_scales": np.log(np.full((3, 3), 0.2, np.float32)),
           "quats": np.array([[1, 0.9, 0.8], [0, 0.1, 0.0], [0, 0.0, 0.3], [0, 0.2, 0.1]], np.float32),
           "logits": np.array([-1.5, -2.0, -1.0], np.float32), "rgb": np.array([[0.9, 0.1, 0.5]] * 3, np.float32).T}
    sc = syn.concat(big, base)
    n = 1203
    cam = syn.pinhole(64, 48, 60.0)
    m = make_mapper(sc, [cam])
    m.render()
    torch.cuda.synchronize()
    _, ids, ranges = gpu_lists(m)
    for t in range(ranges.shape[0]):
        assert set(range(3)) <= set(ids[ranges[t, 0]:ranges[t, 1]].tolist())
    sa = orr.aos(sc)
    gsp, _ = gpu_view_splats(m, 0, n)
    ref = orr.render_fwd(gsp, sa["rgb"], cam, ids, ranges, 0, 16, 16)
    out = m.frame.view(0)
    ok = ref["flag"] == 0
    assert ok.mean() > 0.99
    assert np.abs(out["color"].cpu().numpy() - ref["color"])[:, ok].max() <= PIX_TOL
    flags = oracle_flags(m, [cam], n, sa["rgb"], 16, 16)
    rg = syn.random_image_grads([cam], 5)
    dC, dD, dA = (masked(rg[k], flags) for k in ("dC", "dD", "dA"))
    m.backward(to_device(dC), to_device(dD), to_device(dA))
    torch.cuda.synchronize()
    g2, grgb = orr.render_bwd(gsp, sa["rgb"], cam, ids, ranges, dC[0], dD[0], dA[0], 0, 16, 16)
    grads = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
             "logits": np.zeros(n), "rgb": grgb}
    orr.project_bwd(sa, cam, g2, grads)
    assert_grads_exact(m.grads, orr.grads_to_planes(grads), n)
