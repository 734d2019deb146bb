"""Pins of the keyframe co-visibility / selection oracle (Sec. III-C): the same
camera sees every point, a camera facing away sees none, a sideways shift in
front of a fronto-parallel wall loses exactly the columns geometry predicts, and
hand-built selections."""
import math

import numpy as np

from oracle import keyframes as ok
from paper_2503_01109_gb300 import synthetic as syn


def _wall(W, H, d, holes=0):
    depth = np.full((H, W), d, np.float32)
    if holes:
        depth.reshape(-1)[::holes] = 0.0
    return depth


def test_same_camera_sees_everything():
    cam = syn.room_camera(64, 48, 60.0, seed=3)
    depth = _wall(64, 48, 2.0, holes=7)
    inside, valid = ok.covisibility(depth, cam, [cam], step=1)
    assert valid == int((depth > 0).sum()) and inside[0] == valid


def test_camera_facing_away_sees_nothing():
    cam = syn.pinhole(64, 48, 60.0)
    back = syn.pinhole(64, 48, 60.0, syn.look_pose([0.0, 0.0, 0.0], math.pi))
    inside, valid = ok.covisibility(_wall(64, 48, 2.0), cam, [back], step=2)
    assert valid == 32 * 24 and inside[0] == 0


def test_sideways_shift_loses_the_predicted_columns():
    # keyframe moved by dx along +x in front of a wall at depth D: a point seen at
    # column x lands at u = x - f dx / D; with f dx / D = 20.25 the columns x >= 20
    # stay inside (u >= -0.25), x <= 19 leave (u <= -1.25)
    W, H, f, D = 64, 48, 60.0, 2.0
    dx = 20.25 * D / f
    cam = syn.pinhole(W, H, f)
    moved = syn.pinhole(W, H, f, np.concatenate([np.eye(3), [[-dx], [0.0], [0.0]]], 1))
    inside, valid = ok.covisibility(_wall(W, H, D), cam, [moved], step=1)
    assert valid == W * H and inside[0] == (W - 20) * H
    # and every other sample with step 4: columns 20, 24, ..., 60 of 0, 4, ..., 60
    inside, valid = ok.covisibility(_wall(W, H, D), cam, [moved], step=4)
    assert valid == 16 * 12 and inside[0] == 11 * 12


def test_points_behind_the_near_plane_are_outside():
    W, H, f = 32, 24, 30.0
    cam = syn.pinhole(W, H, f)
    ahead = syn.pinhole(W, H, f, np.concatenate([np.eye(3), [[0.0], [0.0], [-1.9]]], 1), znear=0.2)
    inside, valid = ok.covisibility(_wall(W, H, 2.0), cam, [ahead], step=1)   # wall at z = 0.1 < znear
    assert inside[0] == 0 and valid == W * H


def test_selection_hand_cases():
    inside = np.array([80, 69, 71, 10, 0, 50, 69], np.int64)
    u = np.array([0.5, 0.9, 0.1, 0.3, 0.2, 0.3, 0.05], np.float32)
    kind = ok.select(inside, 100, u, threshold=0.7, frac=0.3)
    # 80 and 71 exceed 70%, 69 does not (exactly 70 is left out of the hand case: 0.7 has no
    # binary representation, and the float32 threshold is a hair below it); of the 5 others round(1.5) = 2 (halves up) with the
    # smallest draws: keyframe 6 (0.05), keyframe 4 (0.2)
    assert kind.tolist() == [1, 0, 1, 0, 2, 0, 2]
    # nothing valid: none co-visible, round(0.3 * 7) = 2 random: keyframes 6 (0.05) and 2 (0.1)
    assert ok.select(inside, 0, u).tolist() == [0, 0, 2, 0, 0, 0, 2]
    assert ok.select(np.array([90]), 100, np.array([0.4])).tolist() == [1]
    tie = ok.select(np.array([0, 0, 0, 0]), 10, np.array([0.5, 0.5, 0.5, 0.5]), frac=0.5)
    assert tie.tolist() == [2, 2, 0, 0]                                  # equal draws: lower index first
