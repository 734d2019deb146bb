"""GPU parity of the splatting path (projection, binning, blending, adjoint,
loss, regulariser, Adam) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import render as orr
from paper_2503_01109_gb300 import fgs, synthetic as syn
from paper_2503_01109_gb300.mapping import Mapper, render as diff_render

from gpu_helpers import (PIX_TOL, assert_grads_exact, flag_fraction, grad_close, gpu_lists, gpu_view_splats,
                         make_mapper, masked, oracle_flags, tile_origin, to_device)

pytestmark = pytest.mark.gpu

CASES = [
    # (W, H, tile_w, tile_h, batch, n, views)
    (64, 48, 16, 16, 128, 2000, 1),   # the tiny configuration
    (70, 45, 16, 16, 64, 1500, 1),    # ragged in both directions
    (70, 45, 8, 8, 32, 1500, 1),
    (50, 70, 16, 32, 256, 1200, 1),
    (64, 48, 16, 16, 128, 1200, 2),   # two views of different size (second 40x30)
]


def cams_for(W, H, views):
    cams = [syn.pinhole(W, H, 60.0)]
    if views > 1:
        cams.append(syn.pinhole(40, 30, 45.0, syn.look_pose([0.05, -0.02, 0.1], 0.08, 0.02)))
    return cams


def check_supports(gsp, ref, vis, cam, tw, th):
    """The integer radius and tile rect of every visible splat are roundings of the
    FP64 oracle's pre-rounding values moved by at most the float32 error of the
    kernel's arithmetic (ceil(3 sqrt(lambda_max)); the tile bounds of the
    opacity-aware box, clamped to the view; an empty rect). Away from an integer
    boundary that set holds one value, so there the GPU must equal the oracle; near
    one it may take the neighbouring integer, and nothing else."""
    A, B, C = (ref["conic"][vis, k] for k in range(3))
    dc = A * C - B * B
    a, b, c = C / dc, -B / dc, A / dc                 # the dilated 2D covariance
    mid = 0.5 * (a + c)
    lam = mid + np.sqrt(np.maximum(0.0, mid * mid - (a * c - b * b)))
    rf = 3.0 * np.sqrt(lam)
    er = 1e-3 * rf + 1e-6    # lambda's float32 error reaches ~3e-4 relative where mid^2 - det cancels
    r = gsp["radius"][vis]
    assert np.all((r >= np.ceil(rf - er)) & (r <= np.ceil(rf + er))), "radius"
    thr = ref["thr"][vis]
    kk = np.minimum(3.0, np.sqrt(np.maximum(thr, 0.0)))
    ex, ey = kk * np.sqrt(a), kk * np.sqrt(c)
    mx, my = ref["mean2d"][vis, 0], ref["mean2d"][vis, 1]
    tiles_x, tiles_y = -(-cam["width"] // tw), -(-cam["height"] // th)
    bounds = []   # per coordinate: the lowest and highest admissible value
    for val, e, fn, t, lo_clip, hi_clip in (
            ((mx - ex - (tw - 1)) / tw, (2e-3 + 1e-4 * ex) / tw, np.ceil, tw, 0, None),
            ((my - ey - (th - 1)) / th, (2e-3 + 1e-4 * ey) / th, np.ceil, th, 0, None),
            ((mx + ex) / tw, (2e-3 + 1e-4 * ex) / tw, np.floor, tw, None, tiles_x - 1),
            ((my + ey) / th, (2e-3 + 1e-4 * ey) / th, np.floor, th, None, tiles_y - 1)):
        lo, hi = fn(val - e), fn(val + e)
        if lo_clip is not None:
            lo, hi = np.maximum(lo, lo_clip), np.maximum(hi, lo_clip)
        else:
            lo, hi = np.minimum(lo, hi_clip), np.minimum(hi, hi_clip)
        bounds.append((lo, hi))
    (x0l, x0h), (y0l, y0h), (x1l, x1h), (y1l, y1h) = bounds
    near_o = np.abs(255.0 * ref["opacity"][vis] - 1.0) < 1e-5   # thr's sign is decided by 255 o > 1
    can_be_empty = (x0h > x1l) | (y0h > y1l) | (thr < 0) | near_o
    can_be_full = (x0l <= x1h) & (y0l <= y1h) & ((thr >= 0) | near_o)
    rc = gsp["rect"][vis]
    empty = (rc[:, 0] > rc[:, 2]) | (rc[:, 1] > rc[:, 3])
    assert np.all(can_be_empty[empty]), "empty rect"
    full = ~empty
    assert np.all(can_be_full[full]), "non-empty rect"
    for k, (lo, hi) in enumerate(bounds):
        assert np.all((rc[full, k] >= lo[full]) & (rc[full, k] <= hi[full])), f"rect[{k}]"
    # and the unique cases are most of them
    exact = (np.ceil(rf - er) == np.ceil(rf + er))
    assert exact.mean() > 0.99 and np.array_equal(r[exact], ref["radius"][vis][exact])


@pytest.mark.parametrize("W,H,tw,th,bd,n,views", CASES)
def test_projection_matches_oracle(cuda_device, W, H, tw, th, bd, n, views):
    sc = syn.tiny_scene(n, seed=W * 7 + H)
    cams = cams_for(W, H, views)
    m = make_mapper(sc, cams, (tw, th), bd)
    m.render()
    torch.cuda.synchronize()
    sa = orr.aos(sc)
    for v, cam in enumerate(cams):
        ref = orr.project(sa, cam, tw, th)
        gsp, raw = gpu_view_splats(m, v, n)
        vis = ref["radius"] > 0
        assert np.array_equal(vis, gsp["radius"] > 0)
        assert np.abs(gsp["mean2d"][vis] - ref["mean2d"][vis]).max() < 1e-3
        assert np.abs(gsp["depth"][vis] - ref["depth"][vis]).max() < 1e-5
        assert np.abs(gsp["opacity"] - ref["opacity"]).max() < 1e-6
        cn, cr = gsp["conic"][vis], ref["conic"][vis]
        scale = np.abs(cr).max(axis=1, keepdims=True)
        assert (np.abs(cn - cr) / scale).max() < 1e-4
        check_supports(gsp, ref, vis, cam, tw, th)


@pytest.mark.parametrize("W,H,tw,th,bd,n,views", CASES)
def test_bin_sort_bit_exact(cuda_device, W, H, tw, th, bd, n, views):
    """Teacher-forced: the oracle bins the GPU's own float32 depths and rects; the
    sorted (tile, id) lists and the tile ranges must be identical."""
    sc = syn.tiny_scene(n, seed=W * 3 + H)
    cams = cams_for(W, H, views)
    m = make_mapper(sc, cams, (tw, th), bd)
    m.render()
    torch.cuda.synchronize()
    tk, ids, ranges = gpu_lists(m)
    depth = np.stack([m.proj.splat[v, :n, 6].cpu().numpy() for v in range(views)]).astype(np.float32)
    radius = np.stack([m.proj.radius[v, :n].cpu().numpy() for v in range(views)])
    rect = np.stack([m.proj.rect[v, :n].cpu().numpy().view(np.uint16).astype(np.int32) for v in range(views)])
    supp = np.stack([orr.support_f32(m.proj.splat[v, :n].cpu().numpy()) for v in range(views)])
    rt, rids, rranges = orr.bin_sort(cams, tw, th, depth, radius, rect, supp)
    assert len(tk) == len(rt)
    assert np.array_equal(tk, rt)
    assert np.array_equal(ids, rids)
    assert np.array_equal(ranges, rranges)


def test_bin_sort_without_tile_keys(cuda_device):
    """tile_keys NULL: the same ids and ranges, and the ranges give back every
    pair's tile."""
    sc = syn.tiny_scene(3000, seed=9)
    cams = cams_for(96, 64, 2)
    m = make_mapper(sc, cams, (16, 16), 64)
    m.render()
    torch.cuda.synchronize()
    tk, ids, ranges = gpu_lists(m)
    m.ids.fill_(-1)
    m.ranges.fill_(-1)
    fgs.fgs_bin_sort(m.proj, m.g.n, cams, m.til, m.ws_bin, None, m.ids, m.ranges, m.num_pairs, m.status)
    torch.cuda.synchronize()
    P = int(m.num_pairs.item())
    assert P == len(tk) > 1000 and int(m.status.item()) == 0
    assert np.array_equal(m.ids[:P].cpu().numpy(), ids)
    r = m.ranges.cpu().numpy()
    assert np.array_equal(r, ranges)
    tile_of = np.repeat(np.arange(len(r)), r[:, 1] - r[:, 0])
    assert np.array_equal(tile_of, tk.astype(np.int64))


@pytest.mark.parametrize("W,H,tw,th,bd,n,views", CASES)
def test_render_forward_matches_oracle(cuda_device, W, H, tw, th, bd, n, views):
    """Teacher-forced splats: colour, depth, alpha, T and contributor counts per
    pixel within 1e-4 (exact counts) outside the oracle's float32 decision band."""
    sc = syn.tiny_scene(n, seed=W + 11 * H)
    cams = cams_for(W, H, views)
    m = make_mapper(sc, cams, (tw, th), bd)
    m.render()
    torch.cuda.synchronize()
    _, ids, ranges = gpu_lists(m)
    rgb = orr.aos(sc)["rgb"]
    bases = tile_origin(cams, tw, th)
    flagged = total = 0
    for v, cam in enumerate(cams):
        gsp, _ = gpu_view_splats(m, v, n)
        ref = orr.render_fwd(gsp, rgb, cam, ids, ranges, bases[v], tw, th)
        out = m.frame.view(v)
        ok = ref["flag"] == 0
        flagged += int((~ok).sum())
        total += ok.size
        for key in ("depth", "alpha", "t_final"):
            assert np.abs(out[key].cpu().numpy() - ref[key])[ok].max() <= PIX_TOL, key
        assert np.abs(out["color"].cpu().numpy() - ref["color"])[:, ok].max() <= PIX_TOL
        assert np.array_equal(out["n_contrib"].cpu().numpy()[ok], ref["n_contrib"][ok])
    assert flagged <= 0.002 * total


@pytest.mark.parametrize("W,H,tw,th,bd,n,views", CASES[:2])
def test_render_end_to_end_from_fp64(cuda_device, W, H, tw, th, bd, n, views):
    """No teacher forcing: the oracle projects, bins and blends in FP64 itself."""
    sc = syn.tiny_scene(n, seed=5 * W + H)
    cams = cams_for(W, H, views)
    m = make_mapper(sc, cams, (tw, th), bd)
    m.render()
    torch.cuda.synchronize()
    st = orr.render_views(sc, cams, tw, th)
    for v in range(views):
        ref = st["out"][v]
        out = m.frame.view(v)
        err = np.abs(out["color"].cpu().numpy() - ref["color"]).max(axis=0)
        err = np.maximum(err, np.abs(out["depth"].cpu().numpy() - ref["depth"]))
        ok = ref["flag"] == 0
        assert ok.mean() >= 0.998
        assert err[ok].max() <= PIX_TOL
        assert np.median(err) < 1e-5


def _bwd_case(sc, cams, tw, th, bd, seed):
    """Adjoint of the blend and the projection on both sides from the same seeded
    upstream gradients, teacher-forced on the GPU's splats and lists, with the
    upstream gradient of every pixel in the oracle's decision band set to zero on
    both sides (those pixels may take the other branch of a threshold in float32,
    so their terms are the only ones allowed to differ)."""
    n = sc["means"].shape[1]
    m = make_mapper(sc, cams, (tw, th), bd)
    m.render()
    torch.cuda.synchronize()
    sa = orr.aos(sc)
    flags = oracle_flags(m, cams, n, sa["rgb"], tw, th)
    rg = syn.random_image_grads(cams, seed)
    dCs, dDs, dAs = (masked(rg[k], flags) for k in ("dC", "dD", "dA"))
    m.backward(to_device(dCs), to_device(dDs), to_device(dAs))
    torch.cuda.synchronize()
    _, ids, ranges = gpu_lists(m)
    bases = tile_origin(cams, tw, th)
    grads = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
             "logits": np.zeros(n), "rgb": np.zeros((n, 3))}
    for v, cam in enumerate(cams):
        gsp, _ = gpu_view_splats(m, v, n)
        g2, grgb = orr.render_bwd(gsp, sa["rgb"], cam, ids, ranges, dCs[v], dDs[v], dAs[v], bases[v], tw, th)
        grads["rgb"] += grgb
        orr.project_bwd(sa, cam, g2, grads)
    return m, orr.grads_to_planes(grads), flags


@pytest.mark.parametrize("W,H,tw,th,bd,n,views", CASES)
def test_render_backward_matches_oracle(cuda_device, W, H, tw, th, bd, n, views):
    """All 14 parameter gradients, every entry, within 1e-3 relative (floor 1e-3 of
    the largest); decision-band pixels (at most 0.2%) masked on both sides."""
    sc = syn.tiny_scene(n, seed=W + H + 3)
    cams = cams_for(W, H, views)
    m, ref, flags = _bwd_case(sc, cams, tw, th, bd, seed=17)
    assert flag_fraction(flags) <= 0.002
    assert_grads_exact(m.grads, ref, n)


def test_autograd_function_uses_the_adjoint(cuda_device):
    sc = syn.tiny_scene(800, seed=2)
    cams = [syn.pinhole(64, 48, 60.0)]
    m = make_mapper(sc, cams)
    params = m.g.buf.requires_grad_(True)
    C, D, A = diff_render(params, m)
    w = torch.randn_like(C)
    (C * w).sum().backward()
    auto = params.grad.clone()
    m2 = make_mapper(sc, cams)
    m2.render()
    m2.backward(w, torch.zeros_like(m2.frame.depth))
    torch.cuda.synchronize()
    # float atomics accumulate in a different order in the two runs
    bad, _ = grad_close(auto.cpu().numpy(), m2.grads.buf.cpu().numpy(), rel=1e-4)
    assert not bad.any()


@pytest.mark.parametrize("sizes, weights", [
    ([(70, 45), (33, 20)], (0.9, 0.1, 0.1)),      # two views, ragged 32x32 loss tiles
    ([(200, 130)], (0.9, 0.1, 0.1)),              # 7 x 5 tiles: interior tile seams both ways
    ([(70, 45)], (0.9, 0.1, 0.0)),                # no SSIM term: L1 colour and depth only
])
def test_loss_matches_oracle(cuda_device, sizes, weights):
    rng = np.random.default_rng(0)
    cams = [syn.pinhole(w, h, 0.8 * w) for w, h in sizes]
    Cs = [rng.uniform(0, 1, (3, c["height"], c["width"])) for c in cams]
    Cg = [rng.uniform(0, 1, (3, c["height"], c["width"])) for c in cams]
    Ds = [rng.uniform(1, 3, (c["height"], c["width"])) for c in cams]
    Dg = [rng.uniform(1, 3, (c["height"], c["width"])) * (rng.uniform(0, 1, (c["height"], c["width"])) > 0.1)
          for c in cams]
    color, depth = fgs.pack_images(cams, Cs, Ds)
    color_gt, depth_gt = fgs.pack_images(cams, Cg, Dg)
    dC = torch.zeros_like(color)
    dD = torch.zeros_like(depth)
    acc = torch.zeros(1, device="cuda")
    ws = fgs.ws_tensor(fgs.fgs_loss_workspace_size(cams))
    fgs.fgs_loss(cams, color, depth, color_gt, depth_gt, *weights, dC, dD, acc, ws)
    torch.cuda.synchronize()
    Lref, off, offp = 0.0, 0, 0
    for v, c in enumerate(cams):
        H, W = c["height"], c["width"]
        C32 = [x.astype(np.float32) for x in (Cs[v], Ds[v], Cg[v], Dg[v])]
        L, rdC, rdD = orr.loss(*C32, *weights)
        Lref += L
        gdc = dC[off:off + 3 * H * W].cpu().numpy().reshape(3, H, W)
        gdd = dD[offp:offp + H * W].cpu().numpy().reshape(H, W)
        assert np.abs(gdc - rdC).max() <= 1e-4 * np.abs(rdC).max()
        assert np.abs(gdd - rdD).max() <= 1e-6 * np.abs(rdD).max()
        off += 3 * H * W
        offp += H * W
    assert float(acc.item()) == pytest.approx(Lref, rel=1e-5)


def test_scale_reg_and_adam_match_oracle(cuda_device):
    sc = syn.tiny_scene(3000, seed=9)
    g = fgs.GaussianMap.from_scene(sc, capacity=3100)
    grads = g.zeros_like()
    rng = np.random.default_rng(1)
    G = rng.standard_normal((14, 3000)).astype(np.float32) * 1e-3
    grads.buf[:, :3000] = torch.as_tensor(G).cuda()
    acc = torch.zeros(1, device="cuda")
    ws = fgs.ws_tensor(fgs.fgs_scale_reg_workspace_size(g.capacity))
    fgs.fgs_scale_reg(g, 0.01, grads, acc, ws)
    torch.cuda.synchronize()
    val, greg = orr.scale_reg(np.asarray(sc["log_scales"], np.float64).T.copy(), 0.01)
    assert float(acc.item()) == pytest.approx(val, rel=1e-5)
    got = grads.plane("log_scales")[:, :3000].cpu().numpy()
    assert np.abs(got - (G[3:6] + greg.T)).max() < 1e-7
    # two Adam steps from the same state
    m, v = g.zeros_like(), g.zeros_like()
    P = g.buf[:, :3000].cpu().numpy().astype(np.float64)
    Gall = grads.buf[:, :3000].cpu().numpy().astype(np.float64)
    M = np.zeros_like(P); Vv = np.zeros_like(P)
    lr_rows = np.repeat(np.array(fgs.DEFAULT_LR), [3, 3, 4, 1, 3])
    for t in (1, 2):
        fgs.fgs_adam(g, grads, m, v, step=t)
        for r in range(14):
            p, gg, mm, vv = P[r].copy(), Gall[r].copy(), M[r].copy(), Vv[r].copy()
            orr.adam(p, gg, mm, vv, lr_rows[r], 0.9, 0.999, 1e-15, t)
            P[r], M[r], Vv[r] = p, mm, vv
    torch.cuda.synchronize()
    assert np.abs(g.buf[:, :3000].cpu().numpy() - P).max() < 1e-5


def l1_sign_band(color, depth, color_gt, depth_gt, tol_c=1e-5, tol_d=1e-4):
    """Pixels where an L1 term's sign could differ between float32 and FP64
    (|C - C*| or |D - D*| within float32 reach of 0, but not both exactly 0 as on
    pixels no Gaussian reaches in either render): the other decision of the loss."""
    band = ((np.abs(color - color_gt) <= tol_c) & ~((color == 0) & (color_gt == 0))).any(axis=0)
    return band | ((np.abs(depth - depth_gt) <= tol_d) & (depth_gt > 0))


def test_mapping_iteration_tiny_config(cuda_device):
    """The tiny configuration end to end from FP64: L1 colour + L1 depth against a
    second seeded scene's render, one iteration.  Loss value within 1e-4; the
    iteration's image gradient equals the oracle's outside the decision bands of
    the blend and of the L1 signs; the adjoint of that image gradient (bands zeroed
    on both sides) matches the oracle's in every entry."""
    cam = syn.pinhole(64, 48, 60.0)
    sc = syn.tiny_scene(2000, 0)
    tgt = syn.tiny_scene(2000, 1)
    st_t = orr.render_views(tgt, [cam])
    Cg, Dg = st_t["out"][0]["color"].astype(np.float32), st_t["out"][0]["depth"].astype(np.float32)
    # the separate end of the iteration keeps the gradients for inspection (the
    # fused one consumes them; its parity with this path is tested on its own)
    m = make_mapper(sc, [cam], loss_w=(1.0, 1.0, 0.0), reg_w=0.0, fused_tail=False)
    cg, dg = fgs.pack_images([cam], [Cg], [Dg])
    m.set_target(cg, dg)
    m.iteration()
    torch.cuda.synchronize()
    st = orr.render_views(sc, [cam])
    out = st["out"][0]
    L, dC, dD = orr.loss(out["color"], out["depth"], Cg, Dg, 1.0, 1.0, 0.0)
    assert float(m.loss_acc.item()) == pytest.approx(L, rel=1e-4)
    band = (out["flag"] != 0) | l1_sign_band(out["color"], out["depth"], Cg, Dg)
    assert band.mean() <= 0.002
    gdC = m.dC.cpu().numpy().reshape(3, 48, 64)
    gdD = m.dD.cpu().numpy().reshape(48, 64)
    assert np.allclose(gdC[:, ~band], dC[:, ~band], rtol=1e-6, atol=0)
    assert np.allclose(gdD[~band], dD[~band], rtol=1e-6, atol=0)
    (mdC,), (mdD,) = masked([gdC], [band]), masked([gdD], [band])
    m2 = make_mapper(sc, [cam])
    m2.render()
    m2.backward(to_device([mdC]), to_device([mdD]))
    torch.cuda.synchronize()
    (rdC,), (rdD,) = masked([dC], [band]), masked([dD], [band])
    ref = orr.grads_to_planes(orr.backward_views(st, [cam], [rdC.astype(np.float64)], [rdD.astype(np.float64)]))
    assert_grads_exact(m2.grads, ref, 2000)


def test_graph_replay_equals_eager(cuda_device):
    """The iteration with the device-side count is capturable; a replayed graph
    produces the same parameters as eager calls."""
    cam = syn.pinhole(64, 48, 60.0)
    sc = syn.tiny_scene(1500, 3)
    tgt = orr.render_views(syn.tiny_scene(1500, 4), [cam])["out"][0]
    cg, dg = fgs.pack_images([cam], [tgt["color"]], [tgt["depth"]])
    eager = make_mapper(sc, [cam], capacity=2048, use_dc=True)
    eager.set_target(cg, dg)
    graphed = make_mapper(sc, [cam], capacity=2048, use_dc=True)
    graphed.set_target(cg, dg)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            eager.iteration()
            graphed.iteration()
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        graphed.iteration()
    for _ in range(3):
        eager.iteration()
        graph.replay()
    torch.cuda.synchronize()
    assert int(graphed.d_step.item()) == int(eager.d_step.item()) == 5
    assert torch.allclose(graphed.g.buf, eager.g.buf, rtol=1e-4, atol=1e-5)


def test_pair_overflow_sets_status(cuda_device):
    sc = syn.tiny_scene(500, 1)
    cams = [syn.pinhole(64, 48, 60.0)]
    m = make_mapper(sc, cams, pair_capacity=16)
    m.render()
    torch.cuda.synchronize()
    assert int(m.status.item()) & fgs.FGS_DEV_PAIR_OVERFLOW
    assert int(m.num_pairs.item()) > 16
    assert int(m.ranges.abs().sum().item()) == 0


def test_invalid_arguments_are_rejected(cuda_device):
    sc = syn.tiny_scene(10, 1)
    m = make_mapper(sc, [syn.pinhole(64, 48, 60.0)])
    with pytest.raises(fgs.FGSError):
        fgs.fgs_project(m.g, [syn.pinhole(64, 48, 60.0)], fgs.tiling(12, 12, 128), m.proj)
    with pytest.raises(fgs.FGSError):
        fgs.fgs_project(m.g, [syn.pinhole(64, 48, 60.0)] * 17, m.til, m.proj)
    small = fgs.ws_tensor(16)
    with pytest.raises(fgs.FGSError):
        fgs.fgs_bin_sort(m.proj, 10, m.cams, m.til, small, m.tile_keys, m.ids, m.ranges, m.num_pairs, m.status)
