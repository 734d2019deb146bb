"""The learned seeding prior on the device: weights, inference and training.

Not in the paper: an extension of eq11.  An MLP (272 -> 128 -> 128 -> 4, GELU)
predicts a new Gaussian's log-scales and opacity logit from the seed's local
spectrum and depth.  Parameters are FP32 masters with BF16 copies; every GEMM runs
in the library's tensor-core kernels.  Training pairs come from the plain mapping
loop itself: seeds appended by ``fgs_fourier_seed`` and their parameters after a
number of mapping iterations.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import fgs

IN, HID, OUT, OUT_PAD = fgs.PRIOR_IN, fgs.PRIOR_HID, fgs.PRIOR_OUT, 8
SHAPES = {"w1": (HID, IN), "b1": (HID,), "w2": (HID, HID), "b2": (HID,), "w3": (OUT_PAD, HID), "b3": (OUT_PAD,)}


def init_params(seed: int = 0) -> dict:
    """Seeded initial weights: uniform +-1/sqrt(fan_in), zero padding rows/columns,
    and the output bias set to a plain eq11-like starting point (log-scale of a
    1-pixel Gaussian at 2 m and f = 600, logit 0)."""
    rng = np.random.default_rng(seed)

    def u(shape, fan):
        return rng.uniform(-1, 1, shape) / math.sqrt(fan)
    w1 = u((HID, IN), 257)
    w1[:, 257:] = 0.0
    w3 = np.zeros((OUT_PAD, HID))
    w3[:OUT] = u((OUT, HID), HID)
    b3 = np.zeros(OUT_PAD)
    b3[:3] = math.log(2.0 / 600.0)
    return {k: np.asarray(v, np.float32) for k, v in
            {"w1": w1, "b1": u(HID, 257), "w2": u((HID, HID), HID), "b2": u(HID, HID), "w3": w3, "b3": b3}.items()}


def bf16_bits_torch(x: torch.Tensor) -> torch.Tensor:
    """Round-to-nearest-even float32 -> BF16 bit patterns (int16 storage)."""
    return x.to(torch.bfloat16).view(torch.int16)


class PriorMLP:
    def __init__(self, params: dict | None = None, device="cuda"):
        params = params or init_params(0)
        self.device = device
        self.master = {k: torch.as_tensor(np.asarray(params[k], np.float32).reshape(SHAPES[k])).to(device).contiguous()
                       for k in SHAPES}
        self.bf = {k: bf16_bits_torch(self.master[k]).contiguous() for k in ("w1", "w2", "w3")}
        self.bias = {k: self.master[k].clone() for k in ("b1", "b2", "b3")}
        n = fgs.fgs_prior_num_params()
        self.m = torch.zeros(n, dtype=torch.float32, device=device)
        self.v = torch.zeros(n, dtype=torch.float32, device=device)
        self.ws = fgs.ws_tensor(fgs.fgs_prior_train_workspace_size(1), device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.step = 0

    def mlp_struct(self) -> fgs.MLP:
        return fgs.MLP(self.bf["w1"].data_ptr(), self.bias["b1"].data_ptr(), self.bf["w2"].data_ptr(),
                       self.bias["b2"].data_ptr(), self.bf["w3"].data_ptr(), self.bias["b3"].data_ptr())

    def master_struct(self) -> fgs.MLPMaster:
        ms = self.master
        return fgs.MLPMaster(ms["w1"].data_ptr(), ms["b1"].data_ptr(), ms["w2"].data_ptr(), ms["b2"].data_ptr(),
                             ms["w3"].data_ptr(), ms["b3"].data_ptr(), self.m.data_ptr(), self.v.data_ptr())

    def infer(self, features: torch.Tensor, status: torch.Tensor | None = None) -> torch.Tensor:
        """Predictions [n][4]; device errors are or-ed into `status` when given."""
        n = features.shape[0]
        out = torch.zeros(n, OUT, dtype=torch.float32, device=self.device)
        fgs.fgs_prior_infer(self.mlp_struct(), features, n, out, status)
        return out

    def train_step(self, features: torch.Tensor, targets: torch.Tensor, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        """One Adam step on a batch; returns the device loss tensor (batch MSE before the step)."""
        self.step += 1
        self.loss.zero_()
        hp = fgs.TrainParams(float(lr), float(beta1), float(beta2), float(eps), int(self.step))
        fgs.fgs_prior_train(self.mlp_struct(), self.master_struct(), features, targets.contiguous(),
                            features.shape[0], hp, self.loss, self.ws)
        return self.loss

    def params_numpy(self) -> dict:
        return {k: v.detach().cpu().numpy().copy() for k, v in self.master.items()}


def features(rgb: torch.Tensor, depth: torch.Tensor, width: int, height: int, xy: torch.Tensor) -> torch.Tensor:
    n = xy.shape[0]
    out = torch.zeros(n, IN, dtype=torch.int16, device=rgb.device)
    fgs.fgs_prior_features(rgb, depth, width, height, xy.to(torch.int32).contiguous(), n, out)
    return out
