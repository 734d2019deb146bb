"""The RGB-D-sequence-size configuration: one 640x480 (f = 525) view inside the
room, a 200k-Gaussian map, targets rendered from a 300k-Gaussian ground-truth
scene, 100 mapping iterations (eq16 + eq15, Adam).  At iterations 0, 50 and 99
the GPU's step is checked against one oracle step from the same state, teacher-
forced on the GPU's float32 splats, tile lists and image gradient: the render
within 1e-4, the loss value and its image gradient, every entry of the 14
parameter gradients within the 1e-3 relative bound (decision-band pixels zeroed
in the image gradient on both sides), and the Adam update of the GPU's gradients
within 1e-5.  Over the run the loss falls; no end-state parity is asked of 100 chaotic
steps."""
import numpy as np
import pytest
import torch

from oracle import render as orr
from paper_2503_01109_gb300 import fgs, synthetic as syn
from paper_2503_01109_gb300.frames import render_targets
from paper_2503_01109_gb300.mapping import PAPER_LOSS, PAPER_REG

from gpu_helpers import (PIX_TOL, assert_grads_exact, gpu_lists, gpu_view_splats, make_mapper, masked,
                         to_device)

pytestmark = pytest.mark.gpu

W, H, F = 640, 480, 525.0
N_MAP, N_GT = 200_000, 300_000
CHECK = (0, 50, 99)


def _scene_of(buf: np.ndarray, n: int) -> dict:
    out = {}
    for k, (a, b) in fgs.PLANES.items():
        v = np.asarray(buf[a:b, :n], np.float64)
        out[k] = v[0].copy() if b - a == 1 else v.copy()
    return out


def _check_step(m, pre, cam, color_gt, depth_gt):
    n = N_MAP
    _, ids, ranges = gpu_lists(m)
    gsp, _ = gpu_view_splats(m, 0, n)
    sa = orr.aos(_scene_of(pre["p"], n))
    # forward, teacher-forced on the GPU's splats and lists
    ref = orr.render_fwd(gsp, sa["rgb"], cam, ids, ranges)
    out = m.frame.view(0)
    ok = ref["flag"] == 0
    assert ok.mean() > 0.99
    color = out["color"].cpu().numpy()
    depth = out["depth"].cpu().numpy()
    assert np.abs(color - ref["color"])[:, ok].max() <= PIX_TOL
    assert np.abs(depth - ref["depth"])[ok].max() <= PIX_TOL * 10   # depth ~ 2 m: 5e-5 relative
    # eq16 on the GPU's render, plus eq15 on the pre-step log-scales
    L, rdC, rdD = orr.loss(color, depth, color_gt, depth_gt, *PAPER_LOSS)
    reg, greg = orr.scale_reg(sa["log_scales"], PAPER_REG)
    assert float(m.loss_acc.item()) == pytest.approx(L + reg, rel=1e-4)
    gdC = m.dC.cpu().numpy().reshape(3, H, W)
    gdD = m.dD.cpu().numpy().reshape(H, W)
    assert np.abs(gdC - rdC).max() <= 1e-4 * np.abs(rdC).max()
    assert np.abs(gdD - rdD).max() <= 1e-6 * np.abs(rdD).max()
    # adjoint of the blend and the projection from the GPU's image gradient with the
    # decision-band pixels zeroed on both sides, through the C ABI on the pre-step
    # parameters and this step's splats and lists; eq15 on the pre-step log-scales
    (mdC,), (mdD,) = masked([gdC], [~ok]), masked([gdD], [~ok])
    g_pre = fgs.GaussianMap.from_scene(_scene_of(pre["p"], n), capacity=m.g.capacity)
    grads_tf = g_pre.zeros_like()
    grad2d = torch.zeros_like(m.grad2d)
    fgs.fgs_render_bwd(g_pre, m.proj, [cam], m.til, m.ids, m.ranges, m.frame, to_device([mdC]), to_device([mdD]),
                       None, grad2d, grads_tf)
    acc = torch.zeros(1, device="cuda")
    fgs.fgs_scale_reg(g_pre, PAPER_REG, grads_tf, acc, fgs.ws_tensor(fgs.fgs_scale_reg_workspace_size(g_pre.capacity)))
    torch.cuda.synchronize()
    g2, grgb = orr.render_bwd(gsp, sa["rgb"], cam, ids, ranges, mdC.astype(np.float64), mdD.astype(np.float64), None)
    grads = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
             "logits": np.zeros(n), "rgb": grgb}
    orr.project_bwd(sa, cam, g2, grads)
    grads["log_scales"] += greg
    assert_grads_exact(grads_tf, orr.grads_to_planes(grads), n)
    # the Adam step of the GPU's gradients from the pre-step state
    P = np.asarray(pre["p"][:, :n], np.float64).copy()
    M = np.asarray(pre["m"][:, :n], np.float64).copy()
    V = np.asarray(pre["v"][:, :n], np.float64).copy()
    G = m.grads.buf[:, :n].cpu().numpy().astype(np.float64)
    lr_rows = np.repeat(np.array(fgs.DEFAULT_LR), [3, 3, 4, 1, 3])
    for r in range(14):
        p, g, mm, vv = P[r].copy(), G[r].copy(), M[r].copy(), V[r].copy()
        orr.adam(p, g, mm, vv, lr_rows[r], 0.9, 0.999, 1e-15, m.host_step)
        P[r], M[r], V[r] = p, mm, vv
    assert np.abs(m.g.buf[:, :n].cpu().numpy() - P).max() < 1e-5
    assert np.abs(m.m.buf[:, :n].cpu().numpy() - M).max() <= 1e-5 * max(np.abs(M).max(), 1e-12)


def test_rgbd_size_mapping_run_step_parity(cuda_device):
    cam = syn.trajectory(1, seed=100, width=W, height=H, f=F)[0]
    colors, depths = render_targets(syn.room_scene(N_GT, seed=1, kind="gt"), [cam])
    m = make_mapper(syn.room_scene(N_MAP, seed=0, kind="map"), [cam], (16, 16), 128, fused_tail=False)
    m.set_target(colors[0], depths[0])
    color_gt = colors[0].cpu().numpy().reshape(3, H, W)
    depth_gt = depths[0].cpu().numpy().reshape(H, W)
    losses = []
    for it in range(100):
        pre = None
        if it in CHECK:
            pre = {k: t.cpu().numpy().copy() for k, t in (("p", m.g.buf), ("m", m.m.buf), ("v", m.v.buf))}
        m.iteration()
        losses.append(float(m.loss_acc.item()))
        if pre is not None:
            _check_step(m, pre, cam, color_gt, depth_gt)
    m.check_status()
    assert np.isfinite(losses).all()
    assert losses[-1] < losses[0]
