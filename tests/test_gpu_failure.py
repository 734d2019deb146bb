"""Failure detection, re-run determinism and checkpoint / resume on the GPU.

Failures are made on purpose only in forms that end by themselves: non-finite
Gaussian parameters (culled and flagged by the projection) and a grid barrier
that waits for an arrival nothing will make (each CTA gives up after a short
bounded wait and reports FGS_DEV_TIMEOUT); the context stays usable and a normal
iteration follows in the same process."""
import numpy as np
import pytest
import torch

from paper_2503_01109_gb300 import fgs, synthetic as syn
from paper_2503_01109_gb300.mapping import Mapper

pytestmark = pytest.mark.gpu

CAM = syn.pinhole(64, 48, 60.0)


def _mapper(scene, cap=None, **kw):
    return Mapper(fgs.GaussianMap.from_scene(scene, cap, "cuda"), [CAM], fgs.tiling(16, 16, 64), **kw)


def _target():
    t = _mapper(syn.tiny_scene(2000, 1))
    t.render()
    return t.frame.color.clone(), t.frame.depth.clone()


def test_nonfinite_gaussians_are_culled_and_flagged(cuda_device):
    sc = syn.tiny_scene(2000, 0)
    bad = {3: ("means", 0, np.nan), 11: ("quats", None, 0.0), 29: ("rgb", 1, np.inf), 47: ("log_scales", 2, 200.0)}
    broken = {k: np.array(v, copy=True) for k, v in sc.items()}
    culled = {k: np.array(v, copy=True) for k, v in sc.items()}
    for i, (key, row, val) in bad.items():
        if row is None:
            broken[key][:, i] = val
        else:
            broken[key][row, i] = val
        culled["means"][:, i] = (0.0, 0.0, -5.0)      # behind the camera: culled by the near plane
    a, b = _mapper(broken), _mapper(culled)
    for m in (a, b):
        m.render()
    torch.cuda.synchronize()
    assert int(a.status.item()) == fgs.FGS_DEV_NONFINITE
    assert int(b.status.item()) == 0
    assert torch.equal(a.proj.radius[0, list(bad)], torch.zeros(len(bad), dtype=torch.int32, device="cuda"))
    for k in ("color", "depth", "alpha", "t_final", "n_contrib"):
        assert torch.equal(getattr(a.frame, k), getattr(b.frame, k)), k
    with pytest.raises(fgs.FGSError):
        a.check_status()


def test_grid_barrier_completes_and_gives_up(cuda_device):
    ws = torch.zeros(64, dtype=torch.uint8, device="cuda")
    passed = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    fgs.fgs_grid_barrier_probe(8, 8, 1_000_000_000, ws, passed, status)
    torch.cuda.synchronize()
    assert int(passed.item()) == 8 and int(status.item()) == 0
    # one arrival too many expected: every CTA gives up after ~50 ms
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    fgs.fgs_grid_barrier_probe(8, 9, 50_000_000, ws, passed, status)
    t1.record()
    torch.cuda.synchronize()
    assert int(passed.item()) == 8                     # nobody else got through
    assert int(status.item()) == fgs.FGS_DEV_TIMEOUT
    assert 40.0 <= t0.elapsed_time(t1) < 2000.0
    # argument errors come back as INVALID_ARGUMENT before any launch
    with pytest.raises(fgs.FGSError):
        fgs.fgs_grid_barrier_probe(8, 7, 50_000_000, ws, passed, status)
    # the context is still usable: a normal mapping iteration follows
    m = _mapper(syn.tiny_scene(2000, 0))
    m.set_target(*_target())
    m.iteration()
    m.check_status()
    assert torch.isfinite(m.loss_acc).all()


def test_rerun_determinism(cuda_device):
    """Binning, forward and loss are bit-identical across runs (no float atomics);
    the adjoint's float atomics leave last-bit differences only."""
    sc = syn.tiny_scene(3000, 4)
    color, depth = _target()
    runs = []
    for _ in range(2):
        m = _mapper(sc, fused_tail=False)
        m.set_target(color, depth)
        m.render()
        fgs.fgs_memset_async(m.loss_acc)
        fgs.fgs_loss(m.cams, m.frame.color, m.frame.depth, m.color_gt, m.depth_gt, *m.loss_w, m.dC, m.dD,
                     m.loss_acc, m.ws_loss)
        m.backward(m.dC, m.dD)
        torch.cuda.synchronize()
        P = int(m.num_pairs.item())
        runs.append((m.tile_keys[:P].clone(), m.ids[:P].clone(), m.ranges.clone(), m.frame.color.clone(),
                     m.frame.n_contrib.clone(), m.loss_acc.clone(), m.grads.buf.clone()))
    for x, y in zip(runs[0][:6], runs[1][:6]):
        assert torch.equal(x, y)
    ga, gb = runs[0][6].cpu().numpy(), runs[1][6].cpu().numpy()
    assert np.allclose(ga, gb, rtol=1e-5, atol=1e-6 * np.abs(ga).max())


def test_checkpoint_resume(cuda_device, tmp_path):
    """k iterations, save, load into a fresh mapper, k more == 2k iterations in one go
    (up to the adjoint's atomic-order rounding)."""
    sc = syn.tiny_scene(2000, 0)
    color, depth = _target()
    k = 4
    whole = _mapper(sc, cap=2100)
    whole.set_target(color, depth)
    for _ in range(2 * k):
        whole.iteration()
    first = _mapper(sc, cap=2100)
    first.set_target(color, depth)
    for _ in range(k):
        first.iteration()
    path = tmp_path / "map.pt"
    torch.save(first.state_dict(), path)
    resumed = Mapper(fgs.GaussianMap(2100, "cuda"), [CAM], fgs.tiling(16, 16, 64))
    resumed.load_state_dict(torch.load(path))
    resumed.set_target(color, depth)
    for _ in range(k):
        resumed.iteration()
    torch.cuda.synchronize()
    for m in (whole, resumed):
        m.check_status()
    assert resumed.host_step == whole.host_step and int(resumed.d_step.item()) == int(whole.d_step.item())
    assert int(resumed.g.d_n.item()) == int(whole.g.d_n.item())
    # Adam turns the sign of a gradient that the atomics leave near zero into a
    # full step, so a handful of entries may differ by about one learning rate
    for x, y in ((resumed.g.buf, whole.g.buf), (resumed.m.buf, whole.m.buf)):
        close = torch.isclose(x, y, rtol=1e-4, atol=1e-5)
        assert close.float().mean().item() > 0.999


def test_lookback_completes_and_gives_up(cuda_device):
    """The depth sort's decoupled look-back: 300 tiles chained through it sum to
    their index; when the first tile never publishes, every later wait gives up
    after its limit with FGS_DEV_TIMEOUT and the context stays usable."""
    n = 300
    ws = fgs.ws_tensor(fgs.fgs_lookback_probe_workspace_size(n), "cuda")
    sums = torch.full((n, 256), -1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    fgs.fgs_lookback_probe(n, False, 1_000_000_000, ws, sums, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(sums, torch.arange(n, dtype=torch.int32, device="cuda")[:, None].expand(n, 256))
    sums.fill_(-1)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    fgs.fgs_lookback_probe(n, True, 50_000_000, ws, sums, status)
    t1.record()
    torch.cuda.synchronize()
    assert int(status.item()) == fgs.FGS_DEV_TIMEOUT
    assert 40.0 <= t0.elapsed_time(t1) < 2000.0
    assert torch.all(sums[0] == -1)
    with pytest.raises(fgs.FGSError):
        fgs.fgs_lookback_probe(0, False, 50_000_000, ws, sums, status)
    m = _mapper(syn.tiny_scene(2000, 0))
    m.set_target(*_target())
    m.iteration()
    m.check_status()
    assert torch.isfinite(m.loss_acc).all()
