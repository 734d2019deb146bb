"""What the trained prior gains over eq11 alone.  The prior is trained on the
GPU from pairs the plain mapping loop produces (seed features at seeding time,
the seed's parameters after mapping), then evaluated on held-out seeds: its initial
log-scales and opacity must lie closer to the converged parameters than eq11's
(log(d / f) on every axis, logit 0).  The convergence of the loop with and
without the prior is run as well and must not get worse."""
import numpy as np
import pytest
import torch

from paper_2503_01109_gb300 import synthetic as syn
from paper_2503_01109_gb300.convergence import SlamLoop, init_error, opacity_weighted, summarise, train_prior
from paper_2503_01109_gb300.frames import render_targets

pytestmark = pytest.mark.gpu


def test_learned_prior_initialises_closer_to_converged_than_eq11(cuda_device):
    W, H, f = 320, 240, 160.0
    gt = syn.room_scene(200_000, seed=77, kind="gt")
    tr = syn.trajectory(14, seed=41, width=W, height=H, f=f)
    te = syn.trajectory(6, seed=42, width=W, height=H, f=f)
    trc, trd = render_targets(gt, tr)
    tec, ted = render_targets(gt, te)
    rec = SlamLoop(trc, trd, tr, capacity=600_000, target_psnr=1e9, max_iters=40, record_seeds=True)
    rec.run()
    feats, targs = rec.training_pairs(high_only=True)
    assert feats.shape[0] > 2000
    fw, tw = opacity_weighted(feats, targs)
    n = int(0.85 * fw.shape[0])
    prior, hist = train_prior(fw[:n], tw[:n], epochs=10, batch=2048, lr=2e-3)
    assert hist[-1] < hist[0]
    d = fw[n:, 256].to(torch.int32).bitwise_left_shift(16).view(torch.float32)
    err = init_error(prior, fw[n:], tw[n:], d, f)
    assert err["learned"] < 0.8 * err["eq11"], err
    assert err["learned_logit"] < err["eq11_logit"], err
    plain = SlamLoop(tec, ted, te, capacity=600_000, target_psnr=30.0, max_iters=80)
    plain.run()
    learned = SlamLoop(tec, ted, te, capacity=600_000, prior=prior, target_psnr=30.0, max_iters=80)
    learned.run()
    sp, sl = summarise(plain.frames, 30.0), summarise(learned.frames, 30.0)
    assert sl["iters_total"] <= 1.1 * sp["iters_total"], (sp, sl)
