"""GPU parity on scenes built to exercise the rare branches of projection and
blending (see ``synthetic.edge_scene``): Gaussians beyond the Jacobian clamp on
either axis, opacities whose alpha saturates at the 0.99 clamp, means around the
near plane, needle-like Gaussians with nearly degenerate 2D covariances, and
opaque layers that stop pixels early.  Each case is compared with the FP64
oracle element by element: projection, bit-exact lists (teacher-forced), the
forward per pixel outside the decision band, and every entry of every gradient
with the decision-band pixels of the upstream gradient zeroed on both sides."""
import numpy as np
import pytest
import torch

from oracle import render as orr
from paper_2503_01109_gb300 import synthetic as syn

from gpu_helpers import (PIX_TOL, assert_grads_exact, flag_fraction, gpu_lists, gpu_view_splats, make_mapper,
                         masked, oracle_flags, tile_origin, to_device)

pytestmark = pytest.mark.gpu

CASES = [(kind, W, H) for kind in syn.EDGE_KINDS for (W, H) in ((64, 48), (70, 45))]


def _setup(kind, W, H, tw=16, th=16, bd=64):
    sc = syn.edge_scene(kind, 1500, seed=W + H)
    cam = syn.pinhole(W, H, 60.0)
    m = make_mapper(sc, [cam], (tw, th), bd)
    m.render()
    torch.cuda.synchronize()
    return sc, cam, m


@pytest.mark.parametrize("kind,W,H", CASES)
def test_edge_projection_and_lists(cuda_device, kind, W, H):
    sc, cam, m = _setup(kind, W, H)
    n = 1500
    sa = orr.aos(sc)
    ref = orr.project(sa, cam)
    gsp, raw = gpu_view_splats(m, 0, n)
    vis = ref["radius"] > 0
    assert np.array_equal(vis, gsp["radius"] > 0)
    assert np.abs(gsp["mean2d"][vis] - ref["mean2d"][vis]).max() <= 1e-4 * max(1.0, np.abs(ref["mean2d"][vis]).max())
    cn, cr = gsp["conic"][vis], ref["conic"][vis]
    assert (np.abs(cn - cr) / np.abs(cr).max(axis=1, keepdims=True)).max() < 1e-4
    # the branch the case is built for is taken
    u = sa["means"][:, 0] / sa["means"][:, 2]
    v = sa["means"][:, 1] / sa["means"][:, 2]
    if kind == "clamp":
        assert (vis & (np.abs(u) > 1.3 * 0.5 * W / 60.0)).sum() > 100
        assert (vis & (np.abs(v) > 1.3 * 0.5 * H / 60.0)).sum() > 100
    if kind == "near":
        assert ((sa["means"][:, 2] < 0.2) & ~vis).sum() > 50 and ((sa["means"][:, 2] < 0.45) & vis).sum() > 50
    # teacher-forced binning, bit-exact
    tk, ids, ranges = gpu_lists(m)
    rt, rids, rranges = orr.bin_sort([cam], 16, 16, raw[:, 6][None].astype(np.float32),
                                     m.proj.radius[0, :n].cpu().numpy()[None],
                                     m.proj.rect[0, :n].cpu().numpy().view(np.uint16).astype(np.int32)[None],
                                     orr.support_f32(raw)[None])
    assert np.array_equal(tk, rt) and np.array_equal(ids, rids) and np.array_equal(ranges, rranges)


@pytest.mark.parametrize("kind,W,H", CASES)
def test_edge_forward_and_gradients(cuda_device, kind, W, H):
    sc, cam, m = _setup(kind, W, H)
    n = 1500
    sa = orr.aos(sc)
    _, ids, ranges = gpu_lists(m)
    gsp, _ = gpu_view_splats(m, 0, n)
    ref = orr.render_fwd(gsp, sa["rgb"], cam, ids, ranges, 0, 16, 16)
    out = m.frame.view(0)
    ok = ref["flag"] == 0
    assert (~ok).mean() <= 0.005
    for key in ("depth", "alpha", "t_final"):
        assert np.abs(out[key].cpu().numpy() - ref[key])[ok].max() <= PIX_TOL, key
    assert np.abs(out["color"].cpu().numpy() - ref["color"])[:, ok].max() <= PIX_TOL
    assert np.array_equal(out["n_contrib"].cpu().numpy()[ok], ref["n_contrib"][ok])
    if kind in ("opaque", "saturate"):
        assert (ref["t_final"] < 2e-4).sum() > 200          # pixels that stop early
    flags = oracle_flags(m, [cam], n, sa["rgb"], 16, 16)
    assert flag_fraction(flags) <= 0.005
    rg = syn.random_image_grads([cam], W * H)
    dC, dD, dA = (masked(rg[k], flags) for k in ("dC", "dD", "dA"))
    m.backward(to_device(dC), to_device(dD), to_device(dA))
    torch.cuda.synchronize()
    g2, grgb = orr.render_bwd(gsp, sa["rgb"], cam, ids, ranges, dC[0], dD[0], dA[0], 0, 16, 16)
    grads = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
             "logits": np.zeros(n), "rgb": grgb}
    orr.project_bwd(sa, cam, g2, grads)
    ref_g = orr.grads_to_planes(grads)
    assert_grads_exact(m.grads, ref_g, n)
    contrib = np.abs(grgb).sum(1) > 0
    if kind == "clamp":
        u = np.abs(sa["means"][:, 0] / sa["means"][:, 2]) > 1.3 * 0.5 * W / 60.0
        v = np.abs(sa["means"][:, 1] / sa["means"][:, 2]) > 1.3 * 0.5 * H / 60.0
        assert (contrib & u).sum() > 50 and (contrib & v).sum() > 50
    if kind == "saturate":
        o = 1.0 / (1.0 + np.exp(-sa["logits"]))
        assert (contrib & (o > 0.995)).sum() > 100
    if kind == "near":
        assert (contrib & (sa["means"][:, 2] < 0.45)).sum() > 50
