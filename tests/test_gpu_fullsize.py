"""Parity at the benchmark's full size and launch configuration: the 1M-Gaussian
room map, a 1200x680 (f = 600) frame of the benchmark trajectory, 16x16 tiles
with batch depth 128.  Teacher-forced on the GPU's float32 splats: the complete
(tile, id) lists bit-exact, every pixel within 1e-4, every gradient within the
1e-3 relative bound."""
import numpy as np
import pytest
import torch

from oracle import render as orr
from paper_2503_01109_gb300 import fgs, synthetic as syn

from gpu_helpers import PIX_TOL, assert_grads_exact, gpu_lists, gpu_view_splats, make_mapper, masked, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    cam = syn.trajectory(1, seed=100, width=1200, height=680, f=600.0)[0]
    scene = syn.room_scene(1_000_000, seed=0, kind="map")
    m = make_mapper(scene, [cam], (16, 16), 128)
    m.render()
    torch.cuda.synchronize()
    return {"cam": cam, "scene": scene, "m": m, "n": 1_000_000}


def test_full_size_key_lists_bit_exact(cuda_device, full):
    m, n, cam = full["m"], full["n"], full["cam"]
    tk, ids, ranges = gpu_lists(m)
    assert len(tk) > 1_000_000
    depth = m.proj.splat[0, :n, 6].cpu().numpy()[None].astype(np.float32)
    radius = m.proj.radius[0, :n].cpu().numpy()[None]
    rect = m.proj.rect[0, :n].cpu().numpy().view(np.uint16).astype(np.int32)[None]
    supp = orr.support_f32(m.proj.splat[0, :n].cpu().numpy())[None]
    rt, rids, rranges = orr.bin_sort([cam], 16, 16, depth, radius, rect, supp)
    assert np.array_equal(tk, rt) and np.array_equal(ids, rids) and np.array_equal(ranges, rranges)


def test_full_size_render_and_gradients(cuda_device, full):
    m, n, cam = full["m"], full["n"], full["cam"]
    _, ids, ranges = gpu_lists(m)
    gsp, _ = gpu_view_splats(m, 0, n)
    sa = orr.aos(full["scene"])
    ref = orr.render_fwd(gsp, sa["rgb"], cam, ids, ranges)
    out = m.frame.view(0)
    ok = ref["flag"] == 0
    assert ok.mean() > 0.99         # hundreds of splats per pixel: about 1% of pixels hold a band decision
    assert np.abs(out["color"].cpu().numpy() - ref["color"])[:, ok].max() <= PIX_TOL
    assert np.abs(out["depth"].cpu().numpy() - ref["depth"])[ok].max() <= PIX_TOL * 10  # depth ~ 2 m: 5e-5 relative
    assert np.abs(out["alpha"].cpu().numpy() - ref["alpha"])[ok].max() <= PIX_TOL
    assert np.array_equal(out["n_contrib"].cpu().numpy()[ok], ref["n_contrib"][ok])
    # upstream gradients with the decision-band pixels zeroed on both sides
    rg = syn.random_image_grads([cam], 7)
    (dC,), (dD,) = masked(rg["dC"], [~ok]), masked(rg["dD"], [~ok])
    m.backward(to_device([dC]), to_device([dD]), None)
    torch.cuda.synchronize()
    g2, grgb = orr.render_bwd(gsp, sa["rgb"], cam, ids, ranges, dC, dD, None)
    grads = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
             "logits": np.zeros(n), "rgb": grgb}
    orr.project_bwd(sa, cam, g2, grads)
    assert_grads_exact(m.grads, orr.grads_to_planes(grads), n)
