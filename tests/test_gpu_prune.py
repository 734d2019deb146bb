"""Gaussian pruning on the GPU against the oracle: the surviving Gaussians and
their Adam moments bit-exact and in the oracle's storage order (removed slots
below the new count filled from the top), with the host count and with the
device count, the degenerate cases, and a mapping iteration after pruning."""
import math

import numpy as np
import pytest
import torch

from oracle import prune as op
from paper_2503_01109_gb300 import fgs, synthetic as syn
from paper_2503_01109_gb300.mapping import Mapper

pytestmark = pytest.mark.gpu


def _random_map(n, cap, seed):
    rng = np.random.default_rng(seed)
    g = fgs.GaussianMap(cap, "cuda", n)
    planes = rng.normal(0.0, 1.0, (14, cap)).astype(np.float32)
    planes[3:6] = rng.normal(-2.0, 1.0, (3, cap))      # some largest scales above e^-0.7
    planes[10] = rng.normal(-3.0, 2.5, cap)            # some opacities below 0.005
    g.buf.copy_(torch.as_tensor(planes))
    g.d_n.fill_(n)
    return g, planes


def _moments(cap, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(2):
        m = fgs.GaussianMap(cap, "cuda")
        m.buf.copy_(torch.as_tensor(rng.normal(0, 1, (14, cap)).astype(np.float32)))
        out.append(m)
    return out


@pytest.mark.parametrize("use_dc", [False, True])
@pytest.mark.parametrize("n,cap", [(100_000, 120_003), (1, 8), (4097, 4097), (1_113_679, 2_200_000)])
def test_prune_matches_oracle(cuda_device, use_dc, n, cap):
    g, planes = _random_map(n, cap, 3)
    m, v = _moments(cap, 4)
    m0, v0 = m.buf.cpu().numpy(), v.buf.cpu().numpy()
    p = fgs.prune_params(0.005, math.exp(-0.7))
    ws = fgs.ws_tensor(fgs.fgs_prune_workspace_size(cap), "cuda")
    kept_d = torch.zeros(1, dtype=torch.int64, device="cuda")
    fgs.fgs_prune(g, m, v, p, ws, kept_d, use_device_count=use_dc)
    torch.cuda.synchronize()
    ref, keep = op.prune(planes, n, p.min_logit, p.max_log_scale)
    k = ref.shape[1]
    assert int(kept_d.item()) == k
    assert int(g.d_n.item()) == (k if use_dc else n)
    out = g.buf.cpu().numpy()
    assert np.array_equal(out[:, :k], ref)
    order = op.fill_order(keep)
    assert np.array_equal(m.buf.cpu().numpy()[:, :k], m0[:, :n][:, order])
    assert np.array_equal(v.buf.cpu().numpy()[:, :k], v0[:, :n][:, order])
    assert np.array_equal(out[:, n:], planes[:, n:])    # columns past the old count untouched


def test_nothing_everything_and_empty(cuda_device):
    cap = 5000
    ws = fgs.ws_tensor(fgs.fgs_prune_workspace_size(cap), "cuda")
    kept = torch.zeros(1, dtype=torch.int64, device="cuda")
    g, planes = _random_map(3000, cap, 5)
    fgs.fgs_prune(g, None, None, fgs.PruneParams(-1e30, 1e30), ws, kept)
    assert int(kept.item()) == 3000 and np.array_equal(g.buf.cpu().numpy(), planes)
    fgs.fgs_prune(g, None, None, fgs.PruneParams(1e30, 1e30), ws, kept, use_device_count=True)
    assert int(kept.item()) == 0 and int(g.d_n.item()) == 0
    g.n = 0
    fgs.fgs_prune(g, None, None, fgs.PruneParams(0.0, 0.0), ws, kept)
    assert int(kept.item()) == 0


def test_argument_errors(cuda_device):
    g, _ = _random_map(10, 16, 6)
    m, _ = _moments(32, 7)
    ws = fgs.ws_tensor(fgs.fgs_prune_workspace_size(16), "cuda")
    kept = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(fgs.FGSError):
        fgs.fgs_prune(g, m, m, fgs.prune_params(), ws, kept)       # other capacity
    with pytest.raises(fgs.FGSError):
        fgs.fgs_prune(g, m, None, fgs.prune_params(), ws, kept)    # one moment only
    with pytest.raises(fgs.FGSError):
        fgs.fgs_prune(g, None, None, fgs.prune_params(), ws[:16], kept)


def test_mapping_continues_after_pruning(cuda_device):
    cam = syn.pinhole(64, 48, 60.0)
    scene = syn.tiny_scene(2000, 0)
    scene["logits"][::3] = -9.0                  # a third nearly transparent
    g = fgs.GaussianMap.from_scene(scene, 2500, "cuda")
    mp = Mapper(g, [cam], fgs.tiling(16, 16, 64), use_device_count=True)
    tgt = syn.tiny_scene(2000, 1)
    ref = Mapper(fgs.GaussianMap.from_scene(tgt, 2000, "cuda"), [cam], fgs.tiling(16, 16, 64))
    ref.render()
    mp.set_target(ref.frame.color, ref.frame.depth)
    mp.iteration()
    mp.prune(fgs.prune_params(0.005, 0.5))
    assert int(g.d_n.item()) < 2000 - 600
    for _ in range(3):
        mp.iteration()
    mp.check_status()
    assert torch.isfinite(mp.loss_acc).all()
