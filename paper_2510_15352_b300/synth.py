"""Seeded synthetic inputs: Gaussian scenes and robot-mounted cameras.

This module is shared by the tests, the benchmark and the CPU oracle's callers.
It holds none of the rendering arithmetic: it only draws random scene
attributes and builds camera poses. Everything is numpy ``default_rng`` with
explicit seeds; the same call always returns the same arrays.

The paper's own scenes (2,500 reconstructed splat scenes, Sec. 1 and Sec. 3.1)
are not available, so these stand in for them, shaped like the paper's
workload: thousands of robots, each with one camera at 640x480 (Sec. 1,
Table 1), many robots per scene (4,096 environments over 128 scenes, Sec. 3.3).

Scene layout (structure of arrays, float32 unless a half type is requested):
  mean          (3, N)  world position, uniform in a 10 x 10 x 3 m box (z up)
  log_scale     (3, N)  i.i.d. normal(-3, 0.5)
  quat          (4, N)  (w, x, y, z) = normalised standard normal 4-vector
  logit_opacity (N,)    standard normal
  sh            (K, 3, N), K = (deg+1)^2, coefficient-major then channel:
                DC uniform in [-sqrt(pi), sqrt(pi)] (the DC range whose
                degree-0 colour is uniform in [0, 1]); higher coefficients
                normal(0, 0.2)
Camera: world->camera 4x4 viewmat (OpenCV axes: x right, y down, z forward)
and intrinsics (fx, fy, cx, cy); pitch = roll = 0, yaw uniform in [0, 2 pi),
position xy uniform in [1, 9]^2.
"""
from __future__ import annotations

import math

import numpy as np

SCENE_BOX = (10.0, 10.0, 3.0)


def make_scene(n: int, sh_degree: int, seed: int = 0) -> dict:
    """One synthetic scene of ``n`` Gaussians with SH degree ``sh_degree``."""
    rng = np.random.default_rng([seed, 0])
    mean = rng.uniform(0.0, 1.0, size=(3, n)) * np.array(SCENE_BOX)[:, None]
    log_scale = rng.normal(-3.0, 0.5, size=(3, n))
    q = rng.normal(size=(4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    logit = rng.normal(0.0, 1.0, size=n)
    K = (sh_degree + 1) ** 2
    sh = np.empty((K, 3, n))
    sh[0] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), size=(3, n))
    if K > 1:
        sh[1:] = rng.normal(0.0, 0.2, size=(K - 1, 3, n))
    return {
        "mean": mean.astype(np.float32),
        "log_scale": log_scale.astype(np.float32),
        "quat": q.astype(np.float32),
        "logit_opacity": logit.astype(np.float32),
        "sh": sh.astype(np.float32),
        "sh_degree": int(sh_degree),
    }


def viewmat_from_pose(pos, yaw: float) -> np.ndarray:
    """World->camera matrix of a level camera at ``pos`` looking along yaw.

    Camera axes in world coordinates: forward (cos y, sin y, 0), right
    (sin y, -cos y, 0), down (0, 0, -1); rows of R are (right, down, forward)
    and t = -R pos.
    """
    f = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    r = np.array([math.sin(yaw), -math.cos(yaw), 0.0])
    d = np.array([0.0, 0.0, -1.0])
    R = np.stack([r, d, f])
    V = np.eye(4)
    V[:3, :3] = R
    V[:3, 3] = -R @ np.asarray(pos, dtype=np.float64)
    return V


def make_cameras(n: int, W: int, H: int, focal: float, height=(0.5, 0.5),
                 seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """``n`` robot cameras: viewmats (n,4,4) and intrinsics (n,4), float32.

    height: (lo, hi) of the uniform camera height (lo == hi for a fixed one).
    """
    rng = np.random.default_rng([seed, 1])
    yaw = rng.uniform(0.0, 2.0 * math.pi, size=n)
    xy = rng.uniform(1.0, 9.0, size=(n, 2))
    h = rng.uniform(height[0], height[1], size=n) if height[1] > height[0] else \
        np.full(n, float(height[0]))
    vm = np.stack([viewmat_from_pose((xy[i, 0], xy[i, 1], h[i]), yaw[i]) for i in range(n)])
    intr = np.tile(np.array([focal, focal, W / 2.0, H / 2.0]), (n, 1))
    return vm.astype(np.float32), intr.astype(np.float32)


# --------------------------------------------------------------- workloads
# small: 1 scene of 20,000 Gaussians, SH degree 0, 8 cameras at 160x120,
#        f = 120, camera height 0.5 m.
# full:  1 scene of 1,000,000 Gaussians, SH degree 3, 1,024 cameras at
#        640x480, f = 480, camera height uniform in [0.3, 1.2] m; with 4,096
#        cameras (the benchmark's batch) or 1,024.

WORKLOADS = {
    "small_20k_8cam_160x120": dict(n=20_000, deg=0, cams=8, W=160, H=120, f=120.0,
                                   height=(0.5, 0.5)),
    "single_1m_sh3_1024cam_640x480": dict(n=1_000_000, deg=3, cams=1024, W=640, H=480,
                                          f=480.0, height=(0.3, 1.2)),
    # the same scene and camera distribution with the paper's 4,096 robots
    "single_1m_sh3_4096cam_640x480": dict(n=1_000_000, deg=3, cams=4096, W=640, H=480,
                                          f=480.0, height=(0.3, 1.2)),
}


def workload(name: str, seed: int = 0, n_cams: int | None = None):
    """(scene, viewmats, intrinsics, W, H) of a named workload."""
    w = WORKLOADS[name]
    scene = make_scene(w["n"], w["deg"], seed)
    vm, it = make_cameras(n_cams or w["cams"], w["W"], w["H"], w["f"], w["height"], seed)
    return scene, vm, it, w["W"], w["H"]


def to_half(scene: dict, geometry: str = "float16", appearance: str = "bfloat16") -> dict:
    """Reduced-precision copy of a scene: mean, log_scale and quat stored as
    ``geometry``, logit_opacity and sh as ``appearance`` ("float16" or
    "bfloat16"; bfloat16 is held as its uint16 bit pattern, rounded to nearest
    even). ``dequantised`` holds the exact float32 values the stored numbers
    represent, which is what a renderer computes with."""
    stored = {"sh_degree": scene["sh_degree"]}
    deq = {"sh_degree": scene["sh_degree"]}
    for keys, kind in ((("mean", "log_scale", "quat"), geometry),
                       (("logit_opacity", "sh"), appearance)):
        for k in keys:
            a = np.ascontiguousarray(scene[k], dtype=np.float32)
            if kind == "float16":
                h = a.astype(np.float16)
                stored[k] = h
                deq[k] = h.astype(np.float32)
            elif kind == "bfloat16":
                u = a.view(np.uint32).astype(np.uint64)
                bits = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
                stored[k] = bits
                deq[k] = (bits.astype(np.uint32) << 16).view(np.float32)
            else:
                raise ValueError(kind)
    stored["dequantised"] = deq
    return stored


def make_batched(n_scenes: int = 32, n_cams: int = 4096, seed: int = 0,
                 n_range=(200_000, 2_000_000), sh_degree: int = 3, zipf: float = 1.1,
                 sizes=((320, 240, 240.0), (640, 480, 480.0)), height=(0.3, 1.2)):
    """Many robots over many scenes of uneven size (the paper's 4,096
    environments over 128 scenes, Sec. 3.3): scene sizes log-uniform in
    ``n_range``; camera i's scene drawn with P(rank k) proportional to
    k^-zipf over a random permutation of the scenes; camera i's resolution
    and focal length alternate through ``sizes`` (W, H, f) by camera index.
    Returns (scenes, scene_of_camera, viewmats, intrinsics, widths, heights)."""
    rng = np.random.default_rng([seed, 2])
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    counts = np.rint(np.exp(rng.uniform(lo, hi, size=n_scenes))).astype(np.int64)
    scenes = [make_scene(int(counts[s]), sh_degree, seed=1000 * seed + s + 1)
              for s in range(n_scenes)]
    perm = rng.permutation(n_scenes)
    p = np.arange(1, n_scenes + 1, dtype=np.float64) ** -zipf
    rank = rng.choice(n_scenes, size=n_cams, p=p / p.sum())
    scene_of = perm[rank].astype(np.int32)
    rng_c = np.random.default_rng([seed, 3])
    yaw = rng_c.uniform(0.0, 2.0 * math.pi, size=n_cams)
    xy = rng_c.uniform(1.0, 9.0, size=(n_cams, 2))
    h = rng_c.uniform(height[0], height[1], size=n_cams)
    vm = np.stack([viewmat_from_pose((xy[i, 0], xy[i, 1], h[i]), yaw[i]) for i in range(n_cams)])
    which = np.arange(n_cams) % len(sizes)
    W = np.array([sizes[k][0] for k in which], dtype=np.int32)
    H = np.array([sizes[k][1] for k in which], dtype=np.int32)
    f = np.array([sizes[k][2] for k in which])
    intr = np.stack([f, f, W / 2.0, H / 2.0], axis=1)
    return scenes, scene_of, vm.astype(np.float32), intr.astype(np.float32), W, H
