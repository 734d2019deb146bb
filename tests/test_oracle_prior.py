"""Pins of the learned-prior oracle: BF16 rounding bit patterns, GELU values,
finite differences of the MLP loss, and closed-form patch features."""
import math

import numpy as np
import pytest

from oracle import prior as op


def test_bf16_round_ties_to_even():
    one = 1.0
    cases = {
        one: one,
        one + 2 ** -8: one,                         # halfway, even (1.0) kept
        one + 3 * 2 ** -8: one + 2 ** -6,           # halfway between 1+2^-7 and 1+2^-6 -> even
        one + 2 ** -8 + 2 ** -20: one + 2 ** -7,    # just above halfway -> up
        -(one + 2 ** -8 + 2 ** -20): -(one + 2 ** -7),
        one + 2 ** -9: one,
        3.0e38: 2.0 ** 127 * (1 + 98 / 128),      # 3e38 = 2^127 * 1.7634: nearest 8-bit mantissa 1 + 98/128
    }
    for x, want in cases.items():
        got = float(op.bf16_round(np.float32(x)))
        assert got == pytest.approx(want, rel=0, abs=abs(want) * 1e-7), (x, got, want)
    assert op.bf16_bits(np.float32(1.0)) == 0x3F80
    assert op.bf16_bits(np.float32(-2.0)) == 0xC000


def test_gelu_values():
    assert op.gelu(np.array(0.0)) == 0.0
    assert op.gelu(np.array(1.0)) == pytest.approx(0.8413447460685429, rel=1e-15)
    assert op.gelu(np.array(-1.0)) == pytest.approx(-0.15865525393145707, rel=1e-14)
    z = np.linspace(-4, 4, 17)
    h = 1e-6
    assert op.gelu_grad(z) == pytest.approx((op.gelu(z + h) - op.gelu(z - h)) / (2 * h), rel=1e-8, abs=1e-10)


def test_mlp_gradients_central_differences():
    """Backward formulas of the MLP (without BF16 rounding) equal central
    differences of its loss."""
    rng = np.random.default_rng(0)
    p = {k: v.astype(np.float64) for k, v in op.init_params(1).items()}
    n = 6
    x = rng.normal(0, 1, (n, op.IN)); x[:, 257:] = 0
    t = rng.normal(0, 1, (n, op.OUT))
    L, g, _ = op.loss_and_grads(p, x, t, emulate_bf16=False)
    h = 1e-6
    for key, idxs in {"w1": [(0, 0), (5, 100), (127, 256)], "b1": [(3,), (64,)], "w2": [(1, 2), (100, 50)],
                      "b2": [(7,)], "w3": [(0, 0), (3, 127)], "b3": [(1,), (3,)]}.items():
        for idx in idxs:
            q = {k: v.copy() for k, v in p.items()}
            q[key][idx] += h
            Lp = op.loss_and_grads(q, x, t, False)[0]
            q[key][idx] -= 2 * h
            Lm = op.loss_and_grads(q, x, t, False)[0]
            assert (Lp - Lm) / (2 * h) == pytest.approx(g[key][idx], rel=1e-6, abs=1e-10), (key, idx)


def test_patch_features_constant_and_clamp():
    """A constant patch has only the DC term 256 c; patches at the border repeat
    the edge pixels (clamp to edge)."""
    gray = np.full((20, 30), 0.25)
    depth = np.full((20, 30), 2.0)
    f = op.patch_features(gray, depth, np.array([[10, 10], [0, 0]]), round_bf16=False)
    assert f[0, 0] == pytest.approx(math.log1p(64.0), rel=1e-12)
    assert np.abs(f[0, 1:256]).max() < 1e-12
    assert f[0, 256] == 2.0 and np.all(f[:, 257:] == 0)
    ramp = np.tile(np.arange(30, dtype=float), (20, 1)) / 30.0
    f2 = op.patch_features(ramp, depth, np.array([[0, 5]]), round_bf16=False)
    cols = np.clip(np.arange(-8, 8), 0, 29)
    P = np.tile(ramp[0, cols], (16, 1))
    F = np.fft.fft2(P)
    assert f2[0, :256] == pytest.approx(np.log1p(np.abs(F)).ravel(), abs=1e-12)
