"""Autotuner: the search space, the batch signature and the JSON cache (CPU),
and a real tuning run whose choice renders the same images (GPU)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2510_15352_b300 import autotune, synth


def test_candidates_cover_the_space():
    c = list(autotune.candidates())
    # layouts (2,1) (4,1) (8,1) x 4 batches x 2 launch forms (8,4) x groups x chunks, the
    # 4 progressive ones (8,1, separate launches) with 3 depth prefixes: 19 x 3 x 3
    assert len(c) == (4 * 3 + 7) * 3 * 3
    assert {x["depth_prefix"] for x in c} == {0, 2048, 8192}
    assert all(x["depth_prefix"] == 0 for x in c
               if x["pixels_per_thread"] != 8 or x["tiles_per_block"] != 1 or x["persistent"])
    assert {x["pixels_per_thread"] for x in c} == {2, 4, 8}
    assert {(x["pixels_per_thread"], x["tiles_per_block"]) for x in c} == {(2, 1), (4, 1), (8, 1), (8, 4)}
    assert {x["comp_batch"] for x in c if x["pixels_per_thread"] == 8 and x["tiles_per_block"] == 1} \
        == {32, 64, 96, 128}
    assert all(x["comp_batch"] == 32 and x["persistent"] == 0
               for x in c if x["pixels_per_thread"] != 8 or x["tiles_per_block"] != 1)


def test_staged_search_space():
    """The search's stages: the compositing knobs with the default pipeline
    knobs (11 candidates), then the pipeline knobs (9), then the depth prefix
    (3 for the progressive layout, 1 otherwise; none when the space lacks it)."""
    best = dict(autotune.DEFAULTS)
    s1 = list(autotune.candidates(None, autotune.STAGES[0], best))
    assert len(s1) == 11 and all(c["camera_group"] == 128 and c["max_chunk_cameras"] == 2048 for c in s1)
    s2 = list(autotune.candidates(None, autotune.STAGES[1], s1[0]))
    assert len(s2) == 9 and all(c["comp_batch"] == s1[0]["comp_batch"] for c in s2)
    prog = dict(best, pixels_per_thread=8, tiles_per_block=1, persistent=0)
    assert len(list(autotune.candidates(None, autotune.STAGES[2], prog))) == 3
    assert len(list(autotune.candidates(None, autotune.STAGES[2], dict(prog, persistent=1)))) == 1
    # a space without the depth prefix has no third stage (nothing is timed twice)
    small = {"pixels_per_thread": (4, 8), "max_chunk_cameras": (8, 24)}
    assert list(autotune.candidates(small, autotune.STAGES[2], prog)) == []


def test_signature_depends_on_the_batch_not_on_order():
    scenes = [synth.make_scene(1000, 1, 0), synth.make_scene(5000, 3, 1)]
    ids = np.array([0, 1, 1, 0])
    W = np.array([64, 128, 64, 128])
    H = np.array([48, 96, 48, 96])
    a = autotune.signature("B300", scenes, ids, W, H)
    assert a == autotune.signature("B300", scenes, ids[::-1], W[::-1], H[::-1])
    assert a != autotune.signature("B300", scenes, ids, W * 2, H)
    assert a != autotune.signature("other", scenes, ids, W, H)


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "c.json")
    assert autotune.load_cache(p) == {}
    autotune.store_cache("k1", {"pixels_per_thread": 4, "ms": 1.5}, p)
    autotune.store_cache("k2", {"pixels_per_thread": 8, "ms": 2.5}, p)
    c = autotune.load_cache(p)
    assert c["k1"]["pixels_per_thread"] == 4 and c["k2"]["ms"] == 2.5
    assert autotune.config_of({"pixels_per_thread": 2, "camera_group": 16,
                               "max_chunk_cameras": 128, "ms": 3}) == {
        "pixels_per_thread": 2, "camera_group": 16, "max_chunk_cameras": 128}


@pytest.mark.gpu
def test_tuning_run_and_cached_choice(tmp_path):
    import torch
    from paper_2510_15352_b300 import gs
    scenes, which, vm, it, Ws, Hs = synth.make_batched(
        n_scenes=3, n_cams=24, seed=9, n_range=(5_000, 30_000), sh_degree=1,
        sizes=((96, 64, 70.0), (64, 48, 50.0)))
    space = {"pixels_per_thread": (4, 8), "camera_group": (8,), "max_chunk_cameras": (8, 24)}
    p = str(tmp_path / "tune.json")
    best = autotune.tune(scenes, which, vm, it, Ws, Hs, space=space, cache_path=p)
    assert len(best["timings"]) == 4 and best["ms"] == min(t[0] for t in best["timings"])
    again = autotune.tune(scenes, which, vm, it, Ws, Hs, space=space, cache_path=p)
    assert again == best  # served from the cache
    outs = []
    for cfg in ({}, autotune.config_of(best)):
        r = gs.Renderer(device=0, **cfg)
        ids = np.array([r.add_scene(s) for s in scenes], dtype=np.int32)[which]
        rgb, d, _, _ = r.render_v(ids, torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda(), Ws, Hs)
        torch.cuda.synchronize()
        outs.append(rgb.cpu().numpy())
        r.close()
    # layouts differ only in float32 rounding of the pixel offsets
    np.testing.assert_allclose(outs[0], outs[1], atol=1e-4)
