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


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and g^2
    at every step (m_t = (1 - b1^t) g, v_t = (1 - b2^t) g^2), so every step moves a
    parameter by lr g / (|g| + eps): five steps move it by 5 lr sign(g) up to eps."""
    p = {"w": np.array([0.5, -1.0, 2.0])}
    g = {"w": np.array([0.25, -3e-3, 7.0])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    for t in range(1, 6):
        p = op.adam_step(p, g, m, v, t, lr=0.01, eps=1e-8)
    want = np.array([0.5, -1.0, 2.0]) - 5 * 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert p["w"] == pytest.approx(want, rel=1e-12, abs=1e-15)


def test_adam_two_steps_hand_values():
    """Two steps with g1 = 0.5, g2 = -0.25 (lr 0.1, b1 0.9, b2 0.999, eps 1e-8),
    worked by hand: step 1 moves by -0.1 * 0.5 / (0.5 + 1e-8); step 2 has
    m = 0.045 - 0.025 = 0.02, m_hat = 0.02 / 0.19 = 0.10526315789473684,
    v = 0.999 * 0.00025 + 0.001 * 0.0625 = 0.00031225,
    v_hat = 0.00031225 / 0.001999 = 0.15620310155077539, sqrt = 0.39522538070166418,
    so it moves by -0.1 * 0.10526315789473684 / (0.39522538070166418 + 1e-8)."""
    p = {"w": np.array([1.0])}
    m = {"w": np.zeros(1)}
    v = {"w": np.zeros(1)}
    p = op.adam_step(p, {"w": np.array([0.5])}, m, v, 1, lr=0.1, eps=1e-8)
    p1 = 1.0 - 0.1 * 0.5 / (0.5 + 1e-8)
    assert p["w"][0] == pytest.approx(p1, rel=1e-15)
    p = op.adam_step(p, {"w": np.array([-0.25])}, m, v, 2, lr=0.1, eps=1e-8)
    assert m["w"][0] == pytest.approx(0.02, rel=1e-14)
    assert v["w"][0] == pytest.approx(0.00031225, rel=1e-14)
    assert p["w"][0] == pytest.approx(p1 - 0.1 * 0.10526315789473684 / (0.39522538070166418 + 1e-8), rel=1e-13)


def test_apply_to_seeds_hand_cases():
    """The prior's use on seeds: high-frequency seeds take the predicted logit
    always and the predicted log-scales only when all three lie within max_dev of
    eq11's; low-frequency seeds keep eq11 entirely.  The boundary is inclusive."""
    ls11 = np.array([[-5.0, -5.0, -5.0, -4.0]] * 3, np.float32)     # eq11: one value on all axes
    lg11 = np.zeros(4, np.float32)
    pred = np.array([[-5.5, -4.6, -5.0, 1.5],      # all within 1.0: accepted
                     [-5.5, -6.5, -5.0, -2.0],     # y 1.5 away: eq11's scales, predicted logit
                     [-5.5, -4.5, -5.0, 3.0],      # low-frequency: untouched
                     [-5.0, -3.0, -4.0, 0.25]],    # 1.0 exactly away on y: inclusive, accepted
                    np.float32)
    hi = np.array([True, True, False, True])
    ls, lg = op.apply_to_seeds(pred, ls11, lg11, hi, 1.0)
    assert ls[:, 0].tolist() == np.float32([-5.5, -4.6, -5.0]).tolist()
    assert ls[:, 1].tolist() == [-5.0, -5.0, -5.0]
    assert ls[:, 2].tolist() == [-5.0, -5.0, -5.0]
    assert ls[:, 3].tolist() == [-5.0, -3.0, -4.0]
    assert lg.tolist() == [1.5, -2.0, 0.0, 0.25]
