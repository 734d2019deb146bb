"""The fused end of a mapping iteration (fgs_project_bwd_adam) against the
separate calls it replaces (fgs_project_bwd, fgs_scale_reg, fgs_adam) on the same
adjoint output: the same geometric gradients, parameters, Adam moments and
regulariser loss, and the RGB gradient and grad2d left zero for the next adjoint.  (Whole iterations are not
compared: the adjoint's atomic sums differ in their last bits from run to run,
and Adam turns sign noise of near-zero gradients into full-size steps.)"""
import numpy as np
import pytest
import torch

from paper_2503_01109_gb300 import fgs, synthetic as syn
from paper_2503_01109_gb300.mapping import Mapper

pytestmark = pytest.mark.gpu


def _setup(use_dc):
    cams = [syn.pinhole(64, 48, 60.0), syn.pinhole(70, 45, 55.0, syn.look_pose([0.1, 0.0, 0.0], 0.05))]
    tgt = Mapper(fgs.GaussianMap.from_scene(syn.tiny_scene(2000, 1), 2000, "cuda"), cams, fgs.tiling(16, 16, 64))
    tgt.render()
    g = fgs.GaussianMap.from_scene(syn.tiny_scene(2000, 0), 2100, "cuda")
    m = Mapper(g, cams, fgs.tiling(16, 16, 64), use_device_count=use_dc)
    m.set_target(tgt.frame.color, tgt.frame.depth)
    rng = np.random.default_rng(3)
    m.m.buf.copy_(torch.as_tensor(rng.normal(0, 1e-3, m.m.buf.shape).astype(np.float32)))
    m.v.buf.copy_(torch.as_tensor(rng.uniform(0, 1e-5, m.v.buf.shape).astype(np.float32)))
    return m


def _adjoint(m):
    m.render()
    fgs.fgs_memset_async(m.loss_acc)
    fgs.fgs_loss(m.cams, m.frame.color, m.frame.depth, m.color_gt, m.depth_gt, *m.loss_w, m.dC, m.dD, m.loss_acc,
                 m.ws_loss)
    fgs.fgs_memset_async(m.grads.buf)
    fgs.fgs_memset_async(m.grad2d)
    fgs.fgs_render_bwd_splats(m.g, m.proj, m.cams, m.til, m.ids, m.ranges, m.frame, m.dC, m.dD, None, m.grad2d,
                              m.grads, m.status, m.use_dc)


@pytest.mark.parametrize("use_dc,reg_w", [(True, 0.01), (False, 0.0), (True, 0.0)])
def test_fused_tail_equals_separate_calls(cuda_device, use_dc, reg_w):
    m = _setup(use_dc)
    for step in (1, 2):
        _adjoint(m)
        snap = {k: t.clone() for k, t in (("p", m.g.buf), ("m", m.m.buf), ("v", m.v.buf), ("g2", m.grad2d),
                                          ("rgb", m.grads.plane("rgb")), ("loss", m.loss_acc))}
        # separate calls
        fgs.fgs_project_bwd(m.g, m.proj, m.cams, m.grad2d, m.grads, m.use_dc)
        if reg_w:
            fgs.fgs_scale_reg(m.g, reg_w, m.grads, m.loss_acc, m.ws_reg, m.use_dc)
        fgs.fgs_adam(m.g, m.grads, m.m, m.v, m.lr, step=step, use_device_count=m.use_dc)
        ref = {k: t.clone() for k, t in (("p", m.g.buf), ("m", m.m.buf), ("v", m.v.buf), ("loss", m.loss_acc),
                                         ("g", m.grads.buf[:11]))}
        # the same inputs through the fused call
        m.g.buf.copy_(snap["p"])
        m.m.buf.copy_(snap["m"])
        m.v.buf.copy_(snap["v"])
        m.grad2d.copy_(snap["g2"])
        m.grads.buf[:11].fill_(123.0)      # stored over, never read
        m.grads.plane("rgb").copy_(snap["rgb"])
        m.loss_acc.copy_(snap["loss"])
        fgs.fgs_project_bwd_adam(m.g, m.proj, m.cams, m.grad2d, m.grads, reg_w, m.loss_acc, m.m, m.v, m.lr,
                                 step=step, ws=m.ws_fused, use_device_count=m.use_dc)
        torch.cuda.synchronize()
        n = m.g.n                              # planes past the live count are not written
        ga, gb = ref["g"][:, :n].cpu().numpy(), m.grads.buf[:11, :n].cpu().numpy()
        assert np.allclose(ga, gb, rtol=1e-6, atol=1e-6 * np.abs(ga).max()), (step, np.abs(ga - gb).max())
        for k in ("p", "m", "v"):
            x0 = snap[k].cpu().numpy().astype(np.float64)
            x = ref[k].cpu().numpy().astype(np.float64)
            y = {"p": m.g.buf, "m": m.m.buf, "v": m.v.buf}[k].cpu().numpy().astype(np.float64)
            # the regulariser's gradient joins the adjoint's in another order, so a
            # gradient may differ in its last bits: the update then agrees to a
            # relative 1e-5 of its own size, and its sum with the old value to a few
            # float32 spacings of the values involved
            big = np.maximum(np.maximum(np.abs(x0), np.abs(x)), np.abs(y)).astype(np.float32)
            tol = 1e-5 * np.abs(x - x0) + 4.0 * np.spacing(big).astype(np.float64)
            bad = np.abs(x - y) > tol
            assert not bad.any(), (step, k, int(bad.sum()), float((np.abs(x - y) / tol).max()))
        assert abs(float(ref["loss"].item()) - float(m.loss_acc.item())) <= 1e-6 * max(abs(float(ref["loss"].item())), 1e-12)
        assert float(m.grads.plane("rgb").abs().max().item()) == 0.0
        assert float(m.grad2d.abs().max().item()) == 0.0
    m.check_status()


def test_fused_tail_full_size(cuda_device):
    """The benchmark's size: the 1M-Gaussian room map at a 1200x680 frame of the
    benchmark trajectory, 16x16 tiles, batch depth 128, device count."""
    from paper_2503_01109_gb300.frames import render_targets
    cam = syn.trajectory(1, seed=100, width=1200, height=680, f=600.0)[0]
    colors, depths = render_targets(syn.room_scene(1_000_000, seed=1000, kind="gt"), [cam])
    g = fgs.GaussianMap.from_scene(syn.room_scene(1_000_000, seed=0, kind="map"), 1_100_000, "cuda")
    m = Mapper(g, [cam], fgs.tiling(16, 16, 128), use_device_count=True)
    m.set_target(colors[0], depths[0])
    _adjoint(m)
    snap = {k: t.clone() for k, t in (("p", m.g.buf), ("m", m.m.buf), ("v", m.v.buf), ("g2", m.grad2d),
                                      ("rgb", m.grads.plane("rgb")), ("loss", m.loss_acc))}
    fgs.fgs_project_bwd(m.g, m.proj, m.cams, m.grad2d, m.grads, True)
    fgs.fgs_scale_reg(m.g, m.reg_w, m.grads, m.loss_acc, m.ws_reg, True)
    fgs.fgs_adam(m.g, m.grads, m.m, m.v, m.lr, step=1, d_step=m.d_step, use_device_count=True)
    torch.cuda.synchronize()
    n = 1_000_000
    ref_g = m.grads.buf[:11, :n].cpu().numpy()
    ref_p, ref_loss = m.g.buf[:, :n].cpu().numpy(), float(m.loss_acc.item())
    m.g.buf.copy_(snap["p"])
    m.m.buf.copy_(snap["m"])
    m.v.buf.copy_(snap["v"])
    m.grad2d.copy_(snap["g2"])
    m.grads.buf.zero_()
    m.grads.plane("rgb").copy_(snap["rgb"])
    m.loss_acc.copy_(snap["loss"])
    m.d_step.zero_()
    fgs.fgs_project_bwd_adam(m.g, m.proj, m.cams, m.grad2d, m.grads, m.reg_w, m.loss_acc, m.m, m.v, m.lr,
                             step=1, d_step=m.d_step, ws=m.ws_fused, use_device_count=True)
    torch.cuda.synchronize()
    m.check_status()
    got_g = m.grads.buf[:11, :n].cpu().numpy()
    assert np.allclose(got_g, ref_g, rtol=1e-6, atol=1e-6 * np.abs(ref_g).max())
    x0 = snap["p"][:, :n].cpu().numpy().astype(np.float64)
    x, y = ref_p.astype(np.float64), m.g.buf[:, :n].cpu().numpy().astype(np.float64)
    big = np.maximum(np.maximum(np.abs(x0), np.abs(x)), np.abs(y)).astype(np.float32)
    tol = 1e-5 * np.abs(x - x0) + 4.0 * np.spacing(big).astype(np.float64)
    assert (np.abs(x - y) <= tol).mean() > 0.9999
    assert abs(float(m.loss_acc.item()) - ref_loss) <= 1e-6 * abs(ref_loss)
    assert float(m.grads.plane("rgb").abs().max().item()) == 0.0
    assert float(m.grad2d.abs().max().item()) == 0.0


def test_mapping_iterations_with_the_fused_tail(cuda_device):
    # a plain adjoint (RenderFn's path) between fused iterations leaves dirty gradients;
    # the next fused iteration clears them first and the loss keeps falling
    m = _setup(True)
    losses = []
    for it in range(12):
        m.iteration()
        losses.append(float(m.loss_acc.item()))
        if it == 5:
            m.render()
            m.backward(m.dC, m.dD)
    m.check_status()
    assert losses[-1] < losses[0]
    assert float(m.grads.plane("rgb").abs().max().item()) == 0.0
