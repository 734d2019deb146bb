"""Pins of the pruning oracle (Sec. III-A, "Gaussian Pruning"): hand-built
Gaussians on both sides of each threshold, the strictness of the comparisons,
the storage order (survivors below the new count stay, removed slots are filled
from the top), and the invariants every result must satisfy."""
import math

import numpy as np

from oracle import prune as op


def _planes(logits, log_scales):
    n = len(logits)
    p = np.zeros((14, n + 3), np.float32)
    p[0, :n] = np.arange(n)                      # means.x = original index, to follow the order
    p[3:6, :n] = np.asarray(log_scales, np.float32).T
    p[10, :n] = logits
    p[:, n:] = 77.0                              # columns past n are not live
    return p, n


def test_hand_cases_on_both_sides_of_each_threshold():
    t_o = np.float32(math.log(0.005 / 0.995))   # opacity 0.005
    t_s = np.float32(math.log(0.5))             # scale 0.5
    below = np.nextafter(t_o, np.float32(-np.inf))
    above = np.nextafter(t_s, np.float32(np.inf))
    ok_s = [-3.0, -3.0, -3.0]
    logits = [0.0, t_o, below, 0.0, 0.0, 0.0, -20.0]
    scales = [ok_s, ok_s, ok_s, [t_s, -3.0, -3.0], [-3.0, -3.0, above], [-3.0, above, -9.0], [1.0, 1.0, 1.0]]
    planes, n = _planes(logits, scales)
    kept, keep = op.prune(planes, n, t_o, t_s)
    # equal to a threshold stays (strict comparisons); one ulp past it goes; both reasons together go
    assert keep.tolist() == [True, True, False, True, False, False, False]
    # three survivors: 0 and 1 stay, removed slot 2 takes survivor 3
    assert kept[0].tolist() == [0.0, 1.0, 3.0]


def test_fill_order_by_hand():
    # K = 4 survivors (0, 3, 5, 6): slot 0 stays, removed slots 1 and 2 take 6 and then 5, slot 3 stays
    keep = np.array([True, False, False, True, False, True, True, False])
    assert op.fill_order(keep).tolist() == [0, 6, 5, 3]
    # the survivors are already packed: nothing moves
    assert op.fill_order(np.array([True, True, False, False])).tolist() == [0, 1]
    # only the last one survives: it moves to slot 0
    assert op.fill_order(np.array([False, False, True])).tolist() == [2]


def test_opacity_threshold_is_the_sigmoid_reading():
    # logit < logit(p) <=> sigmoid(logit) < p, for logits away from the rounding of the threshold
    rng = np.random.default_rng(0)
    lg = rng.normal(-4.0, 2.0, 10_000).astype(np.float32)
    p = 0.005
    keep = op.survivors(np.full((3, lg.size), -3.0, np.float32), lg, math.log(p / (1 - p)), 10.0)
    sig = 1.0 / (1.0 + np.exp(-lg.astype(np.float64)))
    far = np.abs(sig - p) > 1e-9
    assert np.array_equal(keep[far], (sig >= p)[far])


def test_invariants_and_order_on_random_maps():
    rng = np.random.default_rng(1)
    n = 5000
    planes = rng.normal(0.0, 1.0, (14, n + 100)).astype(np.float32)
    planes[0, :n] = np.arange(n)
    planes[3:6] = rng.normal(-3.0, 1.5, (3, n + 100))
    planes[10] = rng.normal(-2.0, 3.0, n + 100)
    t_o, t_s = np.float32(-5.0), np.float32(-1.0)
    kept, keep = op.prune(planes, n, t_o, t_s)
    assert kept.shape == (14, int(keep.sum()))
    assert 0 < kept.shape[1] < n
    assert np.all(kept[10] >= t_o) and np.all(kept[3:6].max(axis=0) <= t_s)
    gone = planes[:, :n][:, ~keep]
    assert np.all((gone[10] < t_o) | (gone[3:6].max(axis=0) > t_s))
    k = kept.shape[1]
    src = kept[0].astype(np.int64)               # means.x holds the original index
    assert np.array_equal(np.sort(src), np.flatnonzero(keep))   # each survivor exactly once
    stay = keep[:k]
    assert np.array_equal(src[stay], np.arange(k)[stay])      # survivors below K do not move
    # the removed slots below K, lowest first, hold the survivors from K on, highest first: a loop
    # that fills each hole with the last survivor not yet moved
    moved = [i for i in range(n - 1, k - 1, -1) if keep[i]]
    expect = np.arange(k)
    for slot in range(k):
        if not keep[slot]:
            expect[slot] = moved.pop(0)
    assert np.array_equal(src, expect)
    assert np.array_equal(kept, planes[:, :n][:, expect])


def test_nothing_and_everything_removed():
    rng = np.random.default_rng(2)
    planes = rng.normal(-3.0, 0.3, (14, 64)).astype(np.float32)
    kept, keep = op.prune(planes, 50, -100.0, 100.0)
    assert keep.all() and np.array_equal(kept, planes[:, :50])
    kept, keep = op.prune(planes, 50, 100.0, 100.0)
    assert not keep.any() and kept.shape == (14, 0)
    kept, keep = op.prune(planes, 0, -100.0, 100.0)
    assert kept.shape == (14, 0)
