"""Autotuner for the batched renderer's launch parameters.

It times real renders of the caller's batch (CUDA events on the render
stream, after a warm-up render) with one context whose launch parameters are
changed between candidates (gs_context_set_config; the scenes are uploaded
once), over:
  pixels_per_thread   2, 4 or 8 -- the compositing layout: each warp of a tile
                      block covers 4x16, 8x16 or 16x16 pixels (the shape of the
                      pixel region over which Gaussians are culled and blended);
  tiles_per_block     1 or 4 -- with 8 pixels per thread, one tile per block or a
                      2x2 quad of tiles sharing the list scan and record staging;
  comp_batch          32, 64, 96 or 128 -- Gaussian records staged per
                      compositing batch (8 pixels per thread, one tile per block);
  persistent          0 or 1 -- binning and compositing as separate launches or
                      as one persistent launch pulling work items from a device
                      queue (8 pixels per thread, one tile per block);
  camera_group        cameras of one scene that share one Gaussian load in the
                      projection kernels (Gaussian batch per projection block);
  max_chunk_cameras   cameras per chunk of the render pipeline;
  depth_prefix        0 (the library's 4,096), 2,048 or 8,192 -- ranks per camera
                      the progressive depth order takes first (8 pixels per
                      thread, one tile per block, separate launches): sparser
                      scenes need deeper lists, denser ones fewer.
The search is staged: first the compositing knobs (layout and batch) with the
default pipeline knobs, then the pipeline knobs (camera group and chunk) with
the best compositing knobs, then the depth order's first-phase depth; the
fastest candidate is kept. Results are cached
in a JSON file keyed by the GPU and a signature of the batch (camera count,
resolutions, scene sizes, SH degrees), so a later run with the same kind of
batch skips the search.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

import numpy as np

DEFAULT_SPACE = {
    "pixels_per_thread": (2, 4, 8),
    "tiles_per_block": (1, 4),
    "comp_batch": (32, 64, 96, 128),
    "persistent": (0, 1),
    "camera_group": (32, 64, 128),
    "max_chunk_cameras": (512, 1024, 2048),
    "depth_prefix": (0, 2048, 8192),
}
# the stages of the search: compositing knobs first, then the pipeline knobs,
# then the depth order's first phase
STAGES = (("pixels_per_thread", "tiles_per_block", "comp_batch", "persistent"),
          ("camera_group", "max_chunk_cameras"), ("depth_prefix",))
DEFAULTS = {"pixels_per_thread": 8, "tiles_per_block": 1, "comp_batch": 32, "persistent": 0,
            "camera_group": 128, "max_chunk_cameras": 2048, "depth_prefix": 0}
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gs_b300_autotune.json")


def signature(gpu: str, scenes, scene_ids, widths, heights) -> str:
    """Key of a batch: GPU, camera count, resolution histogram, the scenes'
    sizes (rounded to 2 significant digits) and SH degrees."""
    res, cnt = np.unique(np.stack([np.asarray(widths), np.asarray(heights)], 1), axis=0,
                         return_counts=True)
    used = sorted(set(int(i) for i in np.asarray(scene_ids).ravel()))
    sizes = [float(f"{scenes[i]['mean'].shape[-1]:.2g}") for i in used]
    degs = sorted(set(int(scenes[i]["sh_degree"]) for i in used))
    desc = {"gpu": gpu, "n": int(len(scene_ids)), "res": res.tolist(), "cnt": cnt.tolist(),
            "sizes": sorted(sizes), "deg": degs}
    return hashlib.sha1(json.dumps(desc, sort_keys=True).encode()).hexdigest()[:16]


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(entry_key: str, entry: dict, path: str = DEFAULT_CACHE) -> None:
    cache = load_cache(path)
    cache[entry_key] = entry
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _distinct(c: dict) -> bool:
    """False for combinations the library runs as another one: quads need 8
    pixels per thread, the batch and the persistent launch are knobs of the
    8-pixel, one-tile layout only (others stage 64 in separate launches), and
    the depth prefix matters only for that layout's separate launches (the
    others order the whole list at once)."""
    ppt, tpb = c.get("pixels_per_thread", 8), c.get("tiles_per_block", 1)
    if tpb == 4 and ppt != 8:
        return False
    if (c.get("comp_batch", 32) != 32 or c.get("persistent", 0)) and (ppt != 8 or tpb != 1):
        return False
    if c.get("depth_prefix", 0) != 0 and (ppt != 8 or tpb != 1 or c.get("persistent", 0)):
        return False
    return True


def candidates(space: dict | None = None, keys=None, base: dict | None = None):
    """Every distinct combination of `keys` of the space (all keys by default),
    the other knobs taken from `base`."""
    space = space or DEFAULT_SPACE
    keys = sorted(k for k in (keys or space) if k in space)
    if not keys:  # a stage none of whose knobs the space holds
        return
    for vals in itertools.product(*(space[k] for k in keys)):
        c = dict(base or {})
        c.update(zip(keys, vals))
        if _distinct(c):
            yield c


def tune(scenes, scene_of_camera, viewmats, intrinsics, widths, heights, device: int = 0,
         space: dict | None = None, repeats: int = 2, cache_path: str | None = DEFAULT_CACHE,
         use_cache: bool = True) -> dict:
    """Best launch configuration for this batch (a dict of gs_config fields),
    with the measured milliseconds of every candidate under "timings"."""
    import torch

    from . import gs
    gpu = torch.cuda.get_device_name(device)
    key = signature(gpu, scenes, scene_of_camera, widths, heights)
    if use_cache and cache_path:
        hit = load_cache(cache_path).get(key)
        if hit is not None:
            return hit
    vm = torch.as_tensor(np.ascontiguousarray(viewmats, dtype=np.float32)).cuda(device)
    it = torch.as_tensor(np.ascontiguousarray(intrinsics, dtype=np.float32)).cuda(device)
    P = int((np.asarray(widths, np.int64) * np.asarray(heights)).sum())
    rgb = torch.empty((P, 3), dtype=torch.float32, device=vm.device)
    depth = torch.empty((P,), dtype=torch.float32, device=vm.device)
    stream = torch.cuda.current_stream(device)
    space = space or DEFAULT_SPACE
    timings = []
    r = gs.Renderer(device=device)
    try:
        ids = np.array([r.add_scene(s) for s in scenes], dtype=np.int32)[scene_of_camera]

        def measure(cand):
            for ms, c in timings:  # the previous stage's choice, already timed
                if c == cand:
                    return ms
            r.set_config(**cand)
            r.render_v(ids, vm, it, widths, heights, rgb, depth, stream=stream)  # warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(repeats):
                r.render_v(ids, vm, it, widths, heights, rgb, depth, stream=stream)
            e1.record(stream)
            r.sync(stream)
            ms = e0.elapsed_time(e1) / repeats
            timings.append((ms, dict(cand)))
            return ms

        best = {k: v for k, v in DEFAULTS.items() if k in space}
        for keys in STAGES:
            stage = [c for c in candidates(space, keys, best)]
            if not stage:
                continue
            ms = [measure(c) for c in stage]
            best = stage[int(np.argmin(ms))]
    finally:
        r.close()
    best_ms, best = min(timings, key=lambda t: t[0])
    entry = dict(best)
    entry["ms"] = best_ms
    entry["timings"] = [[ms, c] for ms, c in timings]
    entry["key"] = key
    if cache_path:
        store_cache(key, entry, cache_path)
    return entry


def config_of(entry: dict) -> dict:
    """The gs_config fields of a tuning result (what Renderer(**...) takes)."""
    return {k: entry[k] for k in DEFAULT_SPACE if k in entry}
