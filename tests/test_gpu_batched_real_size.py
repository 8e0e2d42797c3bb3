"""Parity at the real size of the batched workloads, on sampled cameras.

Batched uneven: 32 scenes of 200k-2M Gaussians (SH degree 3, log-uniform
counts), 4,096 cameras assigned with a Zipf(1.1) law, alternating 320x240 and
640x480, rendered in one call with the benchmark's chunking. Reduced
precision: the same 32 scenes stored as FP16 geometry and BF16 appearance,
all 4,096 cameras at 640x480. In both, 16 cameras drawn with seed 1 are
compared with the FP64 oracle pixel by pixel (on the dequantised attributes
for the half-precision scenes) and no unresolved pixel is allowed.
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
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def batched():
    return synth.make_batched(seed=0)


def _sampled(n):
    return np.sort(np.random.default_rng(1).choice(n, size=16, replace=False))


def _check(orc, scene, vm, it, W, H, rgb, depth, T, tot, cam):
    ref = orc.render(scene, vm, it, W, H, bands=BANDS)
    r = compare_camera(rgb, depth, T, ref)
    assert not r["unresolved"], (int(cam), r)
    for k in ("pixels", "flagged", "resolved_by_alternative"):
        tot[k] = tot.get(k, 0) + r[k]
    return ref


def test_batched_uneven_real_size_sampled(torch, orc, batched):
    from paper_2510_15352_b300 import gs
    scenes, which, vm, it, Ws, Hs = batched
    r = gs.Renderer(device=0)  # default chunking and camera groups, as benchmarked
    try:
        sids = [r.add_scene(s) for s in scenes]
        rgb, depth, T, off = r.render_v([sids[k] for k in which], torch.from_numpy(vm).cuda(),
                                        torch.from_numpy(it).cuda(), Ws, Hs, want_T=True)
        torch.cuda.synchronize()
        tot = {}
        for c in _sampled(len(vm)):
            W, H, o = int(Ws[c]), int(Hs[c]), int(off[c])
            g = [x[o:o + W * H].cpu().numpy() for x in (rgb, depth, T)]
            _check(orc, scenes[which[c]], vm[c], it[c], W, H, g[0].reshape(H, W, 3),
                   g[1].reshape(H, W), g[2].reshape(H, W), tot, c)
        print(f"\nbatched uneven, 16 cameras: {tot}")
    finally:
        r.close()


def test_half_storage_real_size_sampled(torch, orc, batched):
    from paper_2510_15352_b300 import gs
    scenes, which, vm, _, _, _ = batched
    n, W, H = len(vm), 640, 480
    it = np.tile(np.array([480.0, 480.0, W / 2, H / 2], np.float32), (n, 1))
    r = gs.Renderer(device=0)
    try:
        halves = {}
        cams = _sampled(n)
        for k in sorted(set(int(which[c]) for c in cams)):
            halves[k] = synth.to_half(scenes[k])
        sids = {}
        for k, sc in enumerate(scenes):
            h = halves[k] if k in halves else synth.to_half(sc)
            sids[k] = r.add_scene(h)
        rgb, depth, T = r.render(np.array([sids[int(k)] for k in which], np.int32),
                                 torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda(), W, H,
                                 want_T=True)
        torch.cuda.synchronize()
        tot, errs = {}, []
        for c in cams:
            k = int(which[c])
            g = [x[c].cpu().numpy() for x in (rgb, depth, T)]
            _check(orc, halves[k]["dequantised"], vm[c], it[c], W, H, *g, tot, c)
            full = orc.render(scenes[k], vm[c], it[c], W, H)
            e = np.abs(g[0] - full["rgb"]).max(axis=-1)
            errs.append(round(float(np.percentile(e, 99)), 5))
        print(f"\nFP16/BF16 storage, 16 cameras: {tot}; p99 |rgb - oracle(float32 "
              f"attributes)| per camera: {errs}")
    finally:
        r.close()
