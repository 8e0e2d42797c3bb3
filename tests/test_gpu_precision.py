"""Reduced-precision attribute storage: FP16 geometry (mean, log-scale,
quaternion), BF16 appearance (opacity logit, SH), FP32 projection, compositing
and transmittance.

Gated: the GPU render of the half-precision scene against the FP64 oracle run
on the dequantised attributes (the exact values the stored numbers hold), at
the float32 tolerances. Reported, not gated: the difference from the oracle on
the original float32 attributes (the storage error itself).
"""
from __future__ import annotations

import numpy as np
import pytest

from _parity import BANDS, compare_camera
from paper_2510_15352_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def _render(torch, scene, vm, it, W, H):
    from paper_2510_15352_b300 import gs
    r = gs.Renderer(device=0)
    try:
        sid = r.add_scene(scene)
        rgb, depth, T = r.render(sid, torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda(),
                                 W, H, want_T=True)
        torch.cuda.synchronize()
        return rgb.cpu().numpy(), depth.cpu().numpy(), T.cpu().numpy()
    finally:
        r.close()


@pytest.mark.parametrize("geometry,appearance", [("float16", "bfloat16"), ("float16", "float16"),
                                                 ("bfloat16", "bfloat16")])
def test_half_storage_matches_oracle_on_dequantised(torch, orc, geometry, appearance):
    scene, vm, it, W, H = synth.workload("small_20k_8cam_160x120")
    half = synth.to_half(scene, geometry, appearance)
    rgb, depth, T = _render(torch, half, vm, it, W, H)
    worst = 0.0
    for c in range(len(vm)):
        ref = orc.render(half["dequantised"], vm[c], it[c], W, H, bands=BANDS)
        r = compare_camera(rgb[c], depth[c], T[c], ref)
        assert not r["unresolved"], r
        full = orc.render(scene, vm[c], it[c], W, H)
        worst = max(worst, float(np.abs(rgb[c] - full["rgb"]).max()))
    print(f"\n{geometry}/{appearance}: max |rgb - oracle(float32 attributes)| = {worst:.4f}")


def test_half_storage_full_size_sampled(torch, orc):
    scene, vm, it, W, H = synth.workload("single_1m_sh3_1024cam_640x480", n_cams=64)
    half = synth.to_half(scene)
    rgb, depth, T = _render(torch, half, vm, it, W, H)
    errs = []
    for c in (0, 63):
        ref = orc.render(half["dequantised"], vm[c], it[c], W, H, bands=BANDS)
        r = compare_camera(rgb[c], depth[c], T[c], ref)
        assert not r["unresolved"], (c, r)
        full = orc.render(scene, vm[c], it[c], W, H)
        e = np.abs(rgb[c] - full["rgb"]).max(axis=-1)
        errs.append((float(e.mean()), float(np.percentile(e, 99)), float(e.max())))
    print("\nfp16/bf16 vs float32 attributes (mean, p99, max per camera):", errs)
