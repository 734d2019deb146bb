"""Oracle of the Gaussian pruning of Sec. III-A (test infrastructure only).

The paper removes Gaussians that grew too large in some dimension (the mapping
re-seeds the region) and Gaussians whose opacity is below a threshold; it states
neither threshold.  The reading used here: opacity below a minimum, i.e. the
opacity logit below logit(minimum), or the largest of the three scales above a
maximum, i.e. the largest log-scale above log(maximum).  Both comparisons are
strict and are taken on the float32 parameters against float32 thresholds
(the precision the parameters live in), so the decision has one answer.

The paper says nothing about where the survivors are stored.  The reading used
here moves as few of them as there are removed slots to fill: with K survivors,
those already below index K stay where they are, and the removed slots below K,
taken from the lowest up, receive the survivors at or above K, taken from the
highest down (each keeps its Adam moments with it).
"""
from __future__ import annotations

import numpy as np


def survivors(log_scales: np.ndarray, logits: np.ndarray, min_logit: float, max_log_scale: float) -> np.ndarray:
    """Boolean mask of the Gaussians that stay: log_scales [3][n], logits [n]
    (float32), thresholds rounded to float32."""
    ls = np.asarray(log_scales, np.float32)
    lg = np.asarray(logits, np.float32)
    t_o, t_s = np.float32(min_logit), np.float32(max_log_scale)
    low_opacity = lg < t_o
    too_large = ls.max(axis=0) > t_s
    return ~(low_opacity | too_large)


def fill_order(keep: np.ndarray) -> np.ndarray:
    """Source column of each of the K = keep.sum() new columns (the reading in the
    module docstring)."""
    keep = np.asarray(keep, bool)
    k = int(keep.sum())
    order = np.arange(k)
    holes = np.flatnonzero(~keep[:k])                  # removed slots below K, lowest first
    movers = (np.flatnonzero(keep[k:]) + k)[::-1]      # survivors at or above K, highest first
    order[holes] = movers
    return order


def prune(planes: np.ndarray, n: int, min_logit: float, max_log_scale: float):
    """planes [14][capacity] float32 (means 3, log-scales 3, quaternion 4, logit,
    RGB 3) of which the first n are live.  Returns (the new columns [14][kept] in
    their storage order, the mask over the n live columns)."""
    keep = survivors(planes[3:6, :n], planes[10, :n], min_logit, max_log_scale)
    return planes[:, :n][:, fill_order(keep)], keep
