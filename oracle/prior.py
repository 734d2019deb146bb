"""Oracle of the learned seeding prior (test infrastructure only).

The prior is not in the paper; it extends Sec. III-A's eq11 (which fixes a new
Gaussian's radius from the frequency class alone) with a small MLP that predicts
log-scales and an opacity logit from the seed's local spectrum and depth.

Definition (FP64 arithmetic on BF16-rounded operands, so the kernels' only
differences are their FP32 accumulation order):
  features: 16x16 gray patch, top-left (x-8, y-8), clamp to the image; its DFT
            (same DFT as eq2, natural frequency order, row = vertical
            frequency); log(1 + |F|) (256 values), then the depth, then 15
            zeros; rounded to BF16.
  forward : z1 = W1 x + b1, h1 = bf16(gelu(z1)); z2 = W2 h1 + b2,
            h2 = bf16(gelu(z2)); y = W3 h2 + b3 (first 4 rows).
  loss    : mean over the n x 4 outputs of (y - target)^2.
  backward: dy = 2 (y - t) / (4 n) rounded to BF16; dW3 = dy^T h2; dh2 = dy W3;
            dz2 = bf16(dh2 * gelu'(z2)); dW2 = dz2^T h1; dh1 = dz2 W2;
            dz1 = bf16(dh1 * gelu'(z1)); dW1 = dz1^T x; bias gradients are the
            column sums of dy, dz2, dz1.
  Adam on FP32 master weights, then BF16 copies.
  use     : for a high-frequency seed the predicted opacity logit replaces
            eq11's initial logit, and the predicted log-scales replace eq11's
            radius unless one of the three lies further than max_dev from
            eq11's log-scale (then all three stay eq11's: eq11 bounds the
            prediction's scale and says nothing about opacity); low-frequency
            seeds keep eq11's values.  The distance test is taken in float32.
GELU is the erf form x Phi(x); its derivative Phi(x) + x phi(x).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

IN, HID, OUT, OUT_PAD = 272, 128, 4, 8


def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value, ties to even, from the definition: keep
    the upper 16 bits of the float32 pattern after adding 0x7FFF plus the lowest
    kept bit.  Input is first rounded to float32.  Finite inputs only."""
    shape = np.shape(x)
    a = np.array(x, np.float32).reshape(-1)
    b = a.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).reshape(shape)


def bf16_bits(x) -> np.ndarray:
    return (bf16_round(x).view(np.uint32) >> 16).astype(np.uint16)


def from_bits(bits) -> np.ndarray:
    return (np.asarray(bits, np.uint32) << 16).view(np.float32)


def gelu(z):
    return z * 0.5 * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def patch_features(gray: np.ndarray, depth: np.ndarray, xy: np.ndarray, round_bf16: bool = True) -> np.ndarray:
    """Feature rows [n][272] of the seeds xy[n] = (x, y)."""
    H, W = gray.shape
    k = np.arange(16)
    Wd = np.exp(-2j * math.pi * (np.outer(k, k) % 16) / 16.0)
    out = np.zeros((xy.shape[0], IN))
    for r, (x, y) in enumerate(np.asarray(xy)):
        rows = np.clip(np.arange(y - 8, y + 8), 0, H - 1)
        cols = np.clip(np.arange(x - 8, x + 8), 0, W - 1)
        P = np.asarray(gray, np.float64)[np.ix_(rows, cols)]
        F = Wd @ P @ Wd.T
        out[r, :256] = np.log1p(np.abs(F)).ravel()
        out[r, 256] = depth[y, x]
    return bf16_round(out).astype(np.float64) if round_bf16 else out


def init_params(seed: int = 0) -> dict:
    """Seeded initial FP32 master weights (uniform +-1/sqrt(fan_in)), padded rows zero."""
    rng = np.random.default_rng(seed)
    def u(shape, fan):
        return rng.uniform(-1, 1, shape) / math.sqrt(fan)
    w3 = np.zeros((OUT_PAD, HID)); w3[:OUT] = u((OUT, HID), HID)
    b3 = np.zeros(OUT_PAD)
    w1 = u((HID, IN), 257); w1[:, 257:] = 0.0
    return {k: np.asarray(v, np.float32) for k, v in
            {"w1": w1, "b1": u(HID, 257), "w2": u((HID, HID), HID), "b2": u(HID, HID), "w3": w3, "b3": b3}.items()}


def forward(params: dict, x: np.ndarray, emulate_bf16: bool = True) -> dict:
    """Forward pass; returns every intermediate (FP64)."""
    r = bf16_round if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3 = (r(params[k]).astype(np.float64) for k in ("w1", "w2", "w3"))
    b1, b2, b3 = (np.asarray(params[k], np.float64) for k in ("b1", "b2", "b3"))
    x = np.asarray(x, np.float64)
    z1 = x @ W1.T + b1
    h1 = r(gelu(z1)).astype(np.float64)
    z2 = h1 @ W2.T + b2
    h2 = r(gelu(z2)).astype(np.float64)
    y = h2 @ W3.T + b3
    return {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "y": y[:, :OUT], "W1": W1, "W2": W2, "W3": W3}


def loss_and_grads(params: dict, x: np.ndarray, target: np.ndarray, emulate_bf16: bool = True):
    """MSE loss and parameter gradients (see module docstring)."""
    r = bf16_round if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    f = forward(params, x, emulate_bf16)
    n = x.shape[0]
    diff = f["y"] - np.asarray(target, np.float64)
    L = float(np.mean(diff * diff))
    dy = np.zeros((n, OUT_PAD))
    dy[:, :OUT] = 2.0 * diff / (OUT * n)
    dy = r(dy).astype(np.float64)
    g = {"w3": dy.T @ f["h2"], "b3": dy.sum(0)}
    dh2 = dy @ f["W3"]
    dz2 = r(dh2 * gelu_grad(f["z2"])).astype(np.float64)
    g["w2"] = dz2.T @ f["h1"]
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ f["W2"]
    dz1 = r(dh1 * gelu_grad(f["z1"])).astype(np.float64)
    g["w1"] = dz1.T @ f["x"]
    g["b1"] = dz1.sum(0)
    return L, g, f


def adam_step(params: dict, grads: dict, m: dict, v: dict, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8) -> dict:
    """Bias-corrected Adam on FP64 copies of the FP32 masters; returns new params."""
    out = {}
    for k in params:
        m[k] = b1 * m[k] + (1 - b1) * grads[k]
        v[k] = b2 * v[k] + (1 - b2) * grads[k] ** 2
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        out[k] = np.asarray(params[k], np.float64) - lr * mh / (np.sqrt(vh) + eps)
    return out


def apply_to_seeds(pred, log_scales_eq11, logits_eq11, is_high, max_dev):
    """The learned prior's initialisation of freshly seeded Gaussians (an
    extension of eq11 of Sec. III-A; see the module docstring).

    pred[k][4] (log-scale x, y, z, opacity logit) per seed, log_scales_eq11[3][k]
    and logits_eq11[k] as eq11 wrote them, is_high[k] the frequency class.
    Returns (log_scales[3][k], logits[k]) as float32."""
    pred = np.asarray(pred, np.float32)
    ls = np.array(log_scales_eq11, np.float32, copy=True)
    lg = np.array(logits_eq11, np.float32, copy=True)
    hi = np.asarray(is_high, bool)
    dev = np.abs(pred[:, :3] - ls.T)                      # float32 subtraction and magnitude
    accept = hi & np.all(dev <= np.float32(max_dev), axis=1)
    lg[hi] = pred[hi, 3]
    ls[:, accept] = pred[accept, :3].T
    return ls, lg
