"""GPU parity of the Fourier seeding (Sec. III-A, eq2-eq11) against the oracle:
high-frequency energy within 2e-5 of its maximum, and -- teacher-forced on the
GPU's float32 energy -- bit-exact threshold, masks and seed list, with the
appended Gaussians matching eq11."""
import numpy as np
import pytest
import torch

from oracle import seed as osd
from paper_2503_01109_gb300 import fgs, synthetic as syn
from paper_2503_01109_gb300.mapping import Mapper

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (70, 45), (45, 64), (48, 64), (640, 480), (1200, 680)]  # (45, 64): an odd width


def run_seed(W, H, seed, with_render=True, max_new=50000, capacity=None, prior=None, pose=None, grids=None,
             split=None):
    """split: None = fgs_fourier_seed; "same_stream" / "side_stream" = fgs_fourier_energy
    (on the current stream / on a second one) then fgs_fourier_seed_from_energy."""
    fr = syn.textured_frame(W, H, seed)
    cam = syn.pinhole(W, H, 0.9 * W, pose)
    rr = syn.fake_render(W, H, seed + 1) if with_render else None
    g = fgs.GaussianMap(capacity or (max_new + 10), "cuda", 0)
    rgb = torch.as_tensor(fr["rgb"]).reshape(-1).cuda()
    depth = torch.as_tensor(fr["depth"]).reshape(-1).cuda()
    rc = rd = ra = None
    if with_render:
        rc = torch.as_tensor(rr["color"]).reshape(-1).cuda()
        rd = torch.as_tensor(rr["depth"]).reshape(-1).cuda()
        ra = torch.as_tensor(rr["alpha"]).reshape(-1).cuda()
    prm = fgs.seed_params(max_new=max_new, **(grids or {}))
    ws = fgs.ws_tensor(fgs.fgs_fourier_seed_workspace_size(W, H, max_new))
    mask = torch.zeros(H * W, dtype=torch.uint8, device="cuda")
    energy = torch.zeros(H * W, dtype=torch.float32, device="cuda")
    num_new = torch.zeros(1, dtype=torch.int32, device="cuda")
    thr = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    if split is None:
        fgs.fgs_fourier_seed(rgb, depth, rc, rd, ra, cam, prm, prior, mask, energy, g, num_new, thr, ws, status)
    else:
        main = torch.cuda.current_stream()
        side = torch.cuda.Stream() if split == "side_stream" else main
        side.wait_stream(main)
        with torch.cuda.stream(side):
            fgs.fgs_fourier_energy(rgb, cam, prm, energy, thr, ws)
        main.wait_stream(side)
        fgs.fgs_fourier_seed(rgb, depth, rc, rd, ra, cam, prm, prior, mask, energy, g, num_new, thr, ws, status,
                             from_energy=True)
    torch.cuda.synchronize()
    return {"frame": fr, "cam": cam, "render": rr, "g": g, "mask": mask.view(H, W).cpu().numpy(),
            "energy": energy.view(H, W).cpu().numpy(), "num_new": int(num_new.item()), "threshold": int(thr.item()),
            "status": int(status.item())}


@pytest.mark.parametrize("grids", [dict(m=8, n=8, alpha_h=4.0, alpha_l=4.0), dict(m=2, n=2, alpha_h=1.0, alpha_l=1.0)])
def test_equidistant_seeding_bit_exact(cuda_device, grids):
    # the equidistant densification of the ablation: one grid and one scale for every pixel
    W, H = 640, 480
    out = run_seed(W, H, seed=11, max_new=400_000, grids=grids)
    fr, rr = out["frame"], out["render"]
    ref = osd.seed_frame(fr["rgb"], fr["depth"], out["cam"], rr["color"], rr["depth"], rr["alpha"],
                         max_new=400_000, energy32=out["energy"], **grids)
    k = ref["xy"].shape[0]
    assert out["num_new"] == k and np.array_equal(out["mask"], ref["mask"])
    got = out["g"].to_scene(k)
    assert np.abs(got["means"] - ref["gaussians"]["means"]).max() <= 1e-5 * np.abs(ref["gaussians"]["means"]).max()
    assert np.abs(got["log_scales"] - ref["gaussians"]["log_scales"]).max() <= 1e-5
    s = grids["m"]
    ys, xs = ref["xy"][:, 1], ref["xy"][:, 0]
    assert np.all(xs % s == 0) and np.all(ys % s == 0)       # one grid, whatever the frequency mask says


@pytest.mark.parametrize("W,H", SIZES)
def test_high_frequency_energy_matches_oracle(cuda_device, W, H):
    out = run_seed(W, H, seed=W + H)
    ref = osd.high_frequency_energy(out["frame"]["rgb"], 0.25)
    assert np.abs(out["energy"] - ref).max() <= 2e-5 * ref.max()


@pytest.mark.parametrize("W,H", SIZES)
def test_masks_and_seeds_bit_exact_teacher_forced(cuda_device, W, H):
    out = run_seed(W, H, seed=3 * W + H)
    fr, rr = out["frame"], out["render"]
    ref = osd.seed_frame(fr["rgb"], fr["depth"], out["cam"], rr["color"], rr["depth"], rr["alpha"],
                         energy32=out["energy"])
    assert out["threshold"] == ref["threshold"]
    assert np.array_equal(out["mask"], ref["mask"])
    k = ref["xy"].shape[0]
    assert out["num_new"] == k and out["status"] == 0
    got = out["g"].to_scene(k)
    gr = ref["gaussians"]
    assert np.abs(got["means"] - gr["means"]).max() <= 1e-5 * np.abs(gr["means"]).max()
    assert np.abs(got["log_scales"] - gr["log_scales"]).max() <= 1e-5
    assert np.array_equal(got["rgb"], np.asarray(gr["rgb"], np.float32))
    assert np.array_equal(got["quats"], np.asarray(gr["quats"], np.float32))
    assert np.array_equal(got["logits"], np.asarray(gr["logits"], np.float32))
    assert int(out["g"].d_n.item()) == k


def test_first_frame_seeds_everywhere_and_cap_order(cuda_device):
    out = run_seed(64, 48, seed=5, with_render=False, max_new=60)
    ref = osd.seed_frame(out["frame"]["rgb"], out["frame"]["depth"], out["cam"], energy32=out["energy"], max_new=60)
    assert out["num_new"] == 60 == ref["xy"].shape[0]
    assert np.array_equal(out["mask"], ref["mask"])
    assert (out["mask"] & 4).all()                       # M_m = everything on the first frame
    got = out["g"].to_scene(60)
    assert np.abs(got["means"] - ref["gaussians"]["means"]).max() < 1e-5 * np.abs(ref["gaussians"]["means"]).max()


def test_map_full_sets_status_and_truncates(cuda_device):
    out = run_seed(64, 48, seed=6, with_render=False, max_new=500, capacity=20)
    assert out["status"] & fgs.FGS_DEV_MAP_FULL
    assert out["num_new"] == 20 and int(out["g"].d_n.item()) == 20


def test_constant_frame_has_no_high_frequency_seeds(cuda_device):
    W, H = 64, 48
    g = fgs.GaussianMap(1000, "cuda", 0)
    rgb = torch.full((3 * H * W,), 0.4, device="cuda")
    depth = torch.full((H * W,), 2.0, device="cuda")
    prm = fgs.seed_params(max_new=1000)
    ws = fgs.ws_tensor(fgs.fgs_fourier_seed_workspace_size(W, H, 1000))
    mask = torch.zeros(H * W, dtype=torch.uint8, device="cuda")
    nn = torch.zeros(1, dtype=torch.int32, device="cuda")
    thr = torch.zeros(1, dtype=torch.int32, device="cuda")
    fgs.fgs_fourier_seed(rgb, depth, None, None, None, syn.pinhole(W, H, 60.0), prm, None, mask, None, g, nn, thr, ws)
    torch.cuda.synchronize()
    m = mask.cpu().numpy()
    assert not (m & 1).any() and (m & 2).all()
    assert int(nn.item()) == (W // 8) * (H // 8)        # low-frequency grid only


def test_unsupported_size_is_rejected(cuda_device):
    W, H = 38, 19                                        # prime factor 19
    g = fgs.GaussianMap(10, "cuda", 0)
    t = torch.zeros(3 * W * H, device="cuda")
    ws = fgs.ws_tensor(fgs.fgs_fourier_seed_workspace_size(W, H, 10))
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(fgs.FGSError):
        fgs.fgs_fourier_seed(t, t, None, None, None, syn.pinhole(W, H, 30.0), fgs.seed_params(max_new=10), None,
                             torch.zeros(W * H, dtype=torch.uint8, device="cuda"), None, g, z, z.clone(), ws)


@pytest.mark.parametrize("W,H", [(45, 64), (1200, 680)])
@pytest.mark.parametrize("split", ["same_stream", "side_stream"])
def test_energy_then_seeds_equals_one_call(cuda_device, W, H, split):
    """fgs_fourier_energy followed by fgs_fourier_seed_from_energy (the frame-only half
    on a second stream, as the frame pipeline runs it) gives fgs_fourier_seed's
    outputs bit for bit."""
    ref = run_seed(W, H, seed=5)
    got = run_seed(W, H, seed=5, split=split)
    assert ref["num_new"] > 100 and ref["status"] == 0
    for k in ("num_new", "threshold", "status"):
        assert got[k] == ref[k], k
    assert np.array_equal(got["mask"], ref["mask"]) and np.array_equal(got["energy"], ref["energy"])
    a, b = ref["g"].to_scene(ref["num_new"]), got["g"].to_scene(got["num_new"])
    for name in a:
        assert np.array_equal(a[name], b[name]), name
