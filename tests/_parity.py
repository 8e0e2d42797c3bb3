"""GPU-vs-oracle comparison helpers (test side).

Tolerances: rgb max abs error 2e-3 per channel, depth relative error 1e-3
with denominator max(|D_oracle|, 1e-3), transmittance abs 2e-3 (float32 path
against the FP64 oracle). A pixel that misses them passes only when the
oracle flagged it as meeting a near-threshold decision and one of the
oracle's alternative results (flipped decisions) is within the same tolerances.
"""
from __future__ import annotations

import numpy as np

import oracle as O

TOL_RGB = 2e-3
TOL_DEPTH_REL = 1e-3
TOL_T = 2e-3

# near-threshold bands for the float32 path: tile bounds / cull boundary within
# 2e-3 px (+2e-6 relative), depth order / near plane within 1e-5 m (+1e-6 rel),
# alpha within 1e-3 in ln(alpha) of 1/255, T' within 1e-3 relative of 1e-4.
BANDS = O.Bands(px_abs=2e-3, px_rel=2e-6, z_abs=1e-5, z_rel=1e-6, ln_alpha=1e-3, T_rel=1e-3,
                max_flips=2, max_leaves=32)


def pixel_errors(rgb, depth, T, ref_rgb, ref_depth, ref_T):
    e_rgb = np.abs(rgb - ref_rgb).max(axis=-1)
    e_d = np.abs(depth - ref_depth) / np.maximum(np.abs(ref_depth), 1e-3)
    e_T = np.abs(T - ref_T)
    return e_rgb, e_d, e_T


def compare_camera(gpu_rgb, gpu_depth, gpu_T, ref: dict) -> dict:
    """Compare one camera; returns counts and worst errors (see module doc)."""
    gpu_rgb = np.asarray(gpu_rgb, dtype=np.float64)
    gpu_depth = np.asarray(gpu_depth, dtype=np.float64)
    gpu_T = np.asarray(gpu_T, dtype=np.float64)
    e_rgb, e_d, e_T = pixel_errors(gpu_rgb, gpu_depth, gpu_T, ref["rgb"], ref["depth"], ref["T"])
    ok = (e_rgb <= TOL_RGB) & (e_d <= TOL_DEPTH_REL) & (e_T <= TOL_T)
    H, W = ok.shape
    bad = np.argwhere(~ok)
    resolved = 0
    unresolved = []
    lp, lv = ref["leaf_pix"], ref["leaf_val"]
    for j, i in bad:
        p = j * W + i
        if not (ref["flags"][j, i] & 1):
            unresolved.append((j, i))
            continue
        leaves = lv[lp == p]
        hit = False
        for L in leaves:
            er = np.abs(gpu_rgb[j, i] - L[0:3]).max()
            ed = abs(gpu_depth[j, i] - L[3]) / max(abs(L[3]), 1e-3)
            et = abs(gpu_T[j, i] - L[4])
            if er <= TOL_RGB and ed <= TOL_DEPTH_REL and et <= TOL_T:
                hit = True
                break
        if hit:
            resolved += 1
        else:
            unresolved.append((j, i))
    flagged = ref["flags"] & 1
    clean = (flagged == 0)
    return {
        "pixels": H * W,
        "flagged": int(flagged.sum()),
        "resolved_by_alternative": resolved,
        "unresolved": unresolved,
        "max_rgb_err_unflagged": float(e_rgb[clean].max()) if clean.any() else 0.0,
        "max_depth_rel_err_unflagged": float(e_d[clean].max()) if clean.any() else 0.0,
        "max_rgb_err": float(e_rgb.max()),
    }
