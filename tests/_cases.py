"""Hand-built scenes and cameras for closed-form and edge-case tests.

Test-side helpers only (no rendering arithmetic): they lay out Gaussian
attributes in the scene layout that both the oracle and the CUDA path take.
"""
from __future__ import annotations

import math

import numpy as np

Y00 = 1.0 / (2.0 * math.sqrt(math.pi))  # textbook constant of the degree-0 real SH


def dc_for_colour(c):
    """DC coefficient whose degree-0 colour is c (colour = 0.5 + Y00 * dc)."""
    return (np.asarray(c, dtype=np.float64) - 0.5) / Y00


def scene_from(means, log_scales, quats, logits, colours=None, sh=None, deg=0):
    """Scene dict from per-Gaussian rows (float32, the renderers' input type)."""
    means = np.atleast_2d(np.asarray(means, dtype=np.float64))
    n = means.shape[0]
    ls = np.broadcast_to(np.asarray(log_scales, dtype=np.float64), (n, 3))
    q = np.broadcast_to(np.asarray(quats, dtype=np.float64), (n, 4))
    lo = np.broadcast_to(np.asarray(logits, dtype=np.float64), (n,))
    K = (deg + 1) ** 2
    if sh is None:
        sh = np.zeros((K, 3, n))
        cols = np.broadcast_to(np.asarray(colours if colours is not None else 0.5,
                                          dtype=np.float64), (n, 3))
        sh[0] = dc_for_colour(cols).T
    return {
        "mean": np.ascontiguousarray(means.T, dtype=np.float32),
        "log_scale": np.ascontiguousarray(ls.T, dtype=np.float32),
        "quat": np.ascontiguousarray(q.T, dtype=np.float32),
        "logit_opacity": np.ascontiguousarray(lo, dtype=np.float32),
        "sh": np.ascontiguousarray(sh, dtype=np.float32),
        "sh_degree": deg,
    }


def identity_camera(W, H, fx, fy=None):
    """Camera at the world origin looking along +z (world = camera frame)."""
    fy = fx if fy is None else fy
    return np.eye(4, dtype=np.float32), np.array([fx, fy, W / 2.0, H / 2.0], dtype=np.float32)


def logit(p):
    return math.log(p / (1.0 - p))


def f32(x):
    """Value as the float32 the renderers receive, widened back to double."""
    return float(np.float32(x))
