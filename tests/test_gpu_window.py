"""The persistent window launch equals the separate forward / loss / adjoint
calls on a mixed-resolution view set, replays from a CUDA graph, and the
autotuner returns a valid tiling."""
import numpy as np
import pytest
import torch

from oracle import render as orr
from paper_2503_01109_gb300 import fgs, synthetic as syn
from paper_2503_01109_gb300.mapping import Mapper
from paper_2503_01109_gb300.window import Window, autotune

from gpu_helpers import (assert_grads_exact, flag_fraction, gpu_lists, gpu_view_splats, grad_close, make_mapper,
                         masked, oracle_flags, tile_origin, to_device)

pytestmark = pytest.mark.gpu


def views():
    return [syn.pinhole(70, 45, 60.0), syn.pinhole(64, 48, 55.0, syn.look_pose([0.05, 0.02, 0.1], 0.1, 0.03)),
            syn.pinhole(33, 20, 30.0, syn.look_pose([-0.1, 0.0, 0.0], -0.1, 0.0))]


def targets(cams, seed):
    fr = [syn.textured_frame(c["width"], c["height"], seed + i) for i, c in enumerate(cams)]
    return fgs.pack_images(cams, [f["rgb"] for f in fr], [f["depth"] for f in fr])


@pytest.mark.parametrize("ordered", [False, True])
@pytest.mark.parametrize("tile,batch", [((16, 16), 128), ((8, 8), 32), ((16, 32), 256), ((16, 16), 64)])
def test_window_equals_separate_calls(cuda_device, tile, batch, ordered):
    """ordered: the window claims its tiles in the heaviest-first order of the
    separate render (fgs_tile_order), which changes no value beyond the order of
    the adjoint's float atomics."""
    cams = views()
    sc = syn.tiny_scene(2500, seed=7)
    cg, dg = targets(cams, 3)
    til = fgs.tiling(tile[0], tile[1], batch)
    # separate calls
    ref = Mapper(fgs.GaussianMap.from_scene(sc), cams, til, reg_w=0.0, use_device_count=True)
    ref.set_target(cg, dg)
    ref.render()
    fgs.fgs_memset_async(ref.loss_acc)
    fgs.fgs_loss(cams, ref.frame.color, ref.frame.depth, cg, dg, 0.9, 0.1, 0.1, ref.dC, ref.dD, ref.loss_acc,
                 ref.ws_loss)
    ref.backward(ref.dC, ref.dD)
    # one persistent launch
    win = Window(fgs.GaussianMap.from_scene(sc), cams, til, reg_w=0.0)
    win.set_target(cg, dg)
    fgs.fgs_project(win.g, cams, til, win.proj, win.status, True)
    fgs.fgs_bin_sort(win.proj, win.g.capacity, cams, til, win.ws_bin, win.tile_keys, win.ids, win.ranges,
                     win.num_pairs, win.status)
    for t in (win.grads.buf, win.grad2d, win.loss_acc):
        fgs.fgs_memset_async(t)
    order = ref.tile_order if ordered else None
    fgs.fgs_render_window(win.g, win.proj, cams, til, win.ids, win.ranges, cg, dg, 0.9, 0.1, 0.1, win.frame, win.dC,
                          win.dD, win.grad2d, win.grads, win.loss_acc, win.ws_win, win.status, tile_order=order)
    fgs.fgs_project_bwd(win.g, win.proj, cams, win.grad2d, win.grads, True)
    torch.cuda.synchronize()
    if ordered:
        assert not torch.equal(order.cpu(), torch.arange(ref.n_tiles, dtype=torch.int32))
    assert int(win.status.item()) == 0 and int(ref.status.item()) == 0
    for k in ("color", "depth", "alpha", "t_final"):
        assert torch.equal(getattr(win.frame, k), getattr(ref.frame, k)), k
    assert torch.equal(win.frame.n_contrib, ref.frame.n_contrib)
    assert torch.equal(win.dC, ref.dC) and torch.equal(win.dD, ref.dD)
    assert float(win.loss_acc.item()) == pytest.approx(float(ref.loss_acc.item()), rel=1e-6)
    bad, _ = grad_close(win.grads.buf.cpu().numpy(), ref.grads.buf.cpu().numpy(), rel=1e-4)
    assert not bad.any()


def test_window_gradients_match_oracle(cuda_device):
    """The window iteration against the FP64 oracle on the mixed-resolution window
    (eq16 with SSIM): the persistent launch's images and image gradients, and its
    parameter gradients through the whole chain.  Checked as a chain of exact
    links: (1) the window's images equal the oracle's outside the decision band and
    its loss and image gradient match the oracle's loss of those images; (2) the
    window's parameter gradients equal the separate adjoint calls' on its own image
    gradient; (3) those calls, with the decision-band pixels of the image gradient
    zeroed on both sides, match the oracle's adjoint in every entry."""
    cams = views()
    n = 2000
    sc = syn.tiny_scene(n, seed=11)
    frs = [syn.textured_frame(c["width"], c["height"], 20 + i) for i, c in enumerate(cams)]
    cg, dg = fgs.pack_images(cams, [f["rgb"] for f in frs], [f["depth"] for f in frs])
    til = fgs.tiling(16, 16, 128)
    win = Window(fgs.GaussianMap.from_scene(sc), cams, til, reg_w=0.0, fused_tail=False)
    win.set_target(cg, dg)
    win.iteration()
    torch.cuda.synchronize()
    st = orr.render_views(sc, cams)
    sizes = fgs.image_sizes(cams)
    L, o = 0.0, 0
    gdCs, gdDs = [], []
    for v, f in enumerate(frs):
        H, W = cams[v]["height"], cams[v]["width"]
        ref = st["out"][v]
        got = win.frame.view(v)
        ok = ref["flag"] == 0
        assert np.abs(got["color"].cpu().numpy() - ref["color"])[:, ok].max() <= 1e-4
        assert np.abs(got["depth"].cpu().numpy() - ref["depth"])[ok].max() <= 1e-4
        # eq16 of the window's own images (the loss is a smooth function of them)
        l, rdC, rdD = orr.loss(got["color"].cpu().numpy(), got["depth"].cpu().numpy(), f["rgb"], f["depth"],
                               0.9, 0.1, 0.1)
        L += l
        gdC = win.dC[3 * o:3 * (o + H * W)].cpu().numpy().reshape(3, H, W)
        gdD = win.dD[o:o + H * W].cpu().numpy().reshape(H, W)
        assert np.abs(gdC - rdC).max() <= 1e-4 * np.abs(rdC).max()
        assert np.abs(gdD - rdD).max() <= 1e-6 * np.abs(rdD).max()
        gdCs.append(gdC)
        gdDs.append(gdD)
        o += sizes[v]
    assert float(win.loss_acc.item()) == pytest.approx(L, rel=1e-5)
    # (2) the separate adjoint calls on the same image gradient
    sep = make_mapper(sc, cams, (16, 16), 128)
    sep.render()
    sep.backward(win.dC, win.dD)
    torch.cuda.synchronize()
    bad, _ = grad_close(win.grads.buf[:, :n].cpu().numpy(), sep.grads.buf[:, :n].cpu().numpy(), rel=1e-4)
    assert not bad.any()
    # (3) the separate calls against the oracle, decision-band pixels zeroed
    flags = oracle_flags(sep, cams, n, orr.aos(sc)["rgb"], 16, 16)
    assert flag_fraction(flags) <= 0.002
    mdC, mdD = masked(gdCs, flags), masked(gdDs, flags)
    sep.backward(to_device(mdC), to_device(mdD))
    torch.cuda.synchronize()
    _, ids, ranges = gpu_lists(sep)
    sa = orr.aos(sc)
    grads = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
             "logits": np.zeros(n), "rgb": np.zeros((n, 3))}
    for v, (cam, base) in enumerate(zip(cams, tile_origin(cams, 16, 16))):
        gsp, _ = gpu_view_splats(sep, v, n)
        g2, grgb = orr.render_bwd(gsp, sa["rgb"], cam, ids, ranges, mdC[v], mdD[v], None, base, 16, 16)
        grads["rgb"] += grgb
        orr.project_bwd(sa, cam, g2, grads)
    assert_grads_exact(sep.grads, orr.grads_to_planes(grads), n)


def test_window_graph_replay_and_autotune(cuda_device):
    cams = views()
    sc = syn.tiny_scene(1500, seed=2)
    cg, dg = targets(cams, 9)
    best, table = autotune(fgs.GaussianMap.from_scene(sc, capacity=1600), cams, cg, dg, reps=2)
    assert len(table) == 12 and (best.tile_w, best.tile_h) in [(8, 8), (16, 16), (16, 32)]
    eager = Window(fgs.GaussianMap.from_scene(sc, capacity=1600), cams, best)
    graphed = Window(fgs.GaussianMap.from_scene(sc, capacity=1600), cams, best)
    for w in (eager, graphed):
        w.set_target(cg, dg)
    for _ in range(2):
        eager.iteration()
    graphed.capture(warmup=2)
    for _ in range(3):
        eager.iteration()
        graphed.replay()
    torch.cuda.synchronize()
    assert int(eager.d_step.item()) == int(graphed.d_step.item()) == 5
    assert int(graphed.status.item()) == 0
    assert torch.allclose(graphed.g.buf, eager.g.buf, rtol=1e-4, atol=1e-5)
