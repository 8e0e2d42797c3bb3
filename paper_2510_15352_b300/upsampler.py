"""Training and evaluation of the learned 4x upsampler on renderer pairs.

The upsampler (gs.Upsampler, kernels in csrc/k_upsample.cu) maps a render at a
quarter of the resolution (intrinsics / 4) to the full-resolution image. It is
trained on pairs the renderer itself produces: the same camera pose rendered
at both resolutions. Everything here is orchestration -- choosing poses,
calling the renderer and the upsampler's gradient / Adam entry points, and
measuring PSNR; the arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import gs, synth


def quarter(intr) -> "object":
    """Intrinsics (fx, fy, cx, cy) of the same camera at a quarter of the
    resolution: pixel centres (i + 1/2) map to (i + 1/2) / 4."""
    return intr / 4.0


def init_params(seed: int) -> np.ndarray:
    """He-normal weights for the ReLU layers, zero biases, zero last layer: the
    untrained network is exactly bilinear upsampling."""
    rng = np.random.default_rng([seed, 11])
    shapes = [(32, 6)] + [(32, 32)] * 4 + [(48, 32)]
    parts = []
    for li, (co, ci) in enumerate(shapes):
        W = rng.normal(0.0, math.sqrt(2.0 / (9 * ci)), size=(co, ci, 3, 3))
        if li == len(shapes) - 1:
            W[:] = 0.0
        parts += [W.ravel(), np.zeros(co)]
    flat = np.concatenate(parts).astype(np.float32)
    assert flat.size == gs.Upsampler.n_params
    return flat


def render_pairs(renderer: "gs.Renderer", scene_id: int, viewmats, intrinsics, W: int, H: int,
                 stream=None):
    """(lr_rgb [n][H/4][W/4][3], lr_depth, hr_rgb [n][H][W][3], hr_depth) device tensors."""
    import torch
    vm = torch.as_tensor(np.ascontiguousarray(viewmats, dtype=np.float32)).cuda(renderer.device)
    it = torch.as_tensor(np.ascontiguousarray(intrinsics, dtype=np.float32)).cuda(renderer.device)
    hr, hd, _ = renderer.render(scene_id, vm, it, W, H, stream=stream)
    lr, ld, _ = renderer.render(scene_id, vm, quarter(it), W // 4, H // 4, stream=stream)
    return lr, ld, hr, hd


def psnr(a, b):
    """Per-frame PSNR (dB) of images clamped to [0, 1]: 10 log10(1 / MSE)."""
    import torch
    mse = ((a.clamp(0, 1) - b.clamp(0, 1)) ** 2).flatten(1).mean(1)
    return 10.0 * torch.log10(1.0 / mse.clamp_min(1e-20))


def evaluate(up: "gs.Upsampler", renderer: "gs.Renderer", scene_id: int, viewmats, intrinsics,
             W: int, H: int, batch: int = 64) -> dict:
    """PSNR of the upsampled render and of plain bilinear upsampling (an
    upsampler with zero parameters) against the full-resolution render."""
    import torch
    bil = gs.Upsampler(device=renderer.device)
    try:
        bil.set_params(np.zeros(gs.Upsampler.n_params, np.float32))
        p_net, p_bil = [], []
        for i in range(0, len(viewmats), batch):
            lr, _, hr, _ = render_pairs(renderer, scene_id, viewmats[i:i + batch],
                                        intrinsics[i:i + batch], W, H)
            out, _ = up.forward(lr)
            ob, _ = bil.forward(lr)
            p_net.append(psnr(out, hr))
            p_bil.append(psnr(ob, hr))
        torch.cuda.synchronize(renderer.device)
    finally:
        bil.close()
    pn, pb = torch.cat(p_net).cpu().numpy(), torch.cat(p_bil).cpu().numpy()
    return {"psnr_mean": float(pn.mean()), "psnr_p5": float(np.percentile(pn, 5)),
            "bilinear_psnr_mean": float(pb.mean()), "bilinear_psnr_p5": float(np.percentile(pb, 5)),
            "frames": int(len(pn))}


def train(up: "gs.Upsampler", renderer: "gs.Renderer", scene_ids, W: int, H: int,
          n_pairs: int, seed: int = 100, frames_per_step: int = 8, render_batch: int = 256,
          lr_max: float = 1e-4, lr_min: float = 1e-6, heights=(0.3, 1.2), log=None) -> list:
    """Adam on the mean squared error against the full-resolution render, over
    n_pairs training pairs (poses from camera seeds seed, seed + 1, ...; the
    scene of each batch cycles through scene_ids), frames_per_step frames per
    step, learning rate cosine-decayed from lr_max to lr_min. Returns the loss
    of every step (device tensors read back at the end)."""
    import torch
    steps_total = max(1, n_pairs // frames_per_step)
    fx = W * 0.75  # 640x480 at fx = 480, 320x240 at fx = 240
    losses = []
    step = 0
    b = 0
    while step < steps_total:
        m = min(render_batch, (steps_total - step) * frames_per_step)
        vm, it = synth.make_cameras(m, W, H, fx, heights, seed=seed + b)
        sid = scene_ids[b % len(scene_ids)]
        lr, _, hr, _ = render_pairs(renderer, sid, vm, it, W, H)
        perm = torch.randperm(m, generator=torch.Generator().manual_seed(seed + b)).cuda(lr.device)
        for k in range(0, m - frames_per_step + 1, frames_per_step):
            if step >= steps_total:
                break
            idx = perm[k:k + frames_per_step]
            lrb, hrb = lr.index_select(0, idx).contiguous(), hr.index_select(0, idx).contiguous()
            loss = up.grad(lrb, hrb)
            rate = lr_min + 0.5 * (lr_max - lr_min) * (1 + math.cos(math.pi * step / steps_total))
            up.adam(rate)
            losses.append(loss)
            step += 1
        b += 1
        if log:
            log(f"pairs {step * frames_per_step}: loss {float(losses[-1].item()):.3e}")
    return [float(x) for x in torch.cat(losses).cpu()]


# A scene whose held-out poses upsample below this PSNR (against the full render)
# is rendered at full resolution instead.
PSNR_FLOOR_DB = 35.0


def validate_scenes(up: "gs.Upsampler", renderer: "gs.Renderer", scene_ids, W: int, H: int,
                    n_poses: int = 8, seed: int = 7000) -> dict:
    """Mean PSNR of the upsampled render per scene on `n_poses` held-out poses
    (robot-height cameras, f = 0.75 W; pose seed `seed + k` for the k-th scene)."""
    out = {}
    for k, sid in enumerate(scene_ids):
        vm, it = synth.make_cameras(n_poses, W, H, 0.75 * W, (0.3, 1.2), seed=seed + k)
        out[int(sid)] = evaluate(up, renderer, sid, vm, it, W, H)["psnr_mean"]
    return out


class FallbackPlan:
    """One batch of cameras split by scene quality: cameras of scenes whose
    validation PSNR is below `floor_db` are rendered at full resolution, the
    others at a quarter of the resolution and upsampled. The split, the index
    tensors and the two output buffers are made once; `render` issues the two
    calls on a stream (nothing else), `assemble` scatters both parts into one
    [n][H][W][3] / [n][H][W] pair in camera order."""

    def __init__(self, scene_of_camera, viewmats, intrinsics, W: int, H: int, psnr_by_scene: dict,
                 floor_db: float = PSNR_FLOOR_DB):
        import torch
        ids = np.asarray(scene_of_camera, dtype=np.int32)
        self.W, self.H, self.n = W, H, len(ids)
        self.slow = np.array([psnr_by_scene[int(s)] < floor_db for s in ids], dtype=bool)
        dev = viewmats.device
        self.fast_idx = torch.from_numpy(np.nonzero(~self.slow)[0]).to(dev)
        self.slow_idx = torch.from_numpy(np.nonzero(self.slow)[0]).to(dev)
        self.ids_f, self.ids_s = ids[~self.slow], ids[self.slow]
        self.vm_f = viewmats[self.fast_idx].contiguous()
        self.it_f = intrinsics[self.fast_idx].contiguous()
        self.vm_s = viewmats[self.slow_idx].contiguous()
        self.it_s = intrinsics[self.slow_idx].contiguous()
        f32 = dict(dtype=torch.float32, device=dev)
        self.rgb_f = torch.empty((len(self.ids_f), H, W, 3), **f32)
        self.depth_f = torch.empty((len(self.ids_f), H, W), **f32)
        self.rgb_s = torch.empty((len(self.ids_s), H, W, 3), **f32)
        self.depth_s = torch.empty((len(self.ids_s), H, W), **f32)

    @property
    def fallback_cameras(self) -> int:
        return int(self.slow.sum())

    def render(self, renderer: "gs.Renderer", up: "gs.Upsampler", stream=None) -> None:
        if len(self.ids_f):
            renderer.render_upsampled(up, self.ids_f, self.vm_f, self.it_f, self.W, self.H,
                                      self.rgb_f, self.depth_f, stream=stream)
        if len(self.ids_s):
            renderer.render(self.ids_s, self.vm_s, self.it_s, self.W, self.H, self.rgb_s,
                            self.depth_s, stream=stream)

    def assemble(self, rgb=None, depth=None):
        import torch
        dev = self.rgb_f.device
        if rgb is None:
            rgb = torch.empty((self.n, self.H, self.W, 3), dtype=torch.float32, device=dev)
        if depth is None:
            depth = torch.empty((self.n, self.H, self.W), dtype=torch.float32, device=dev)
        if len(self.ids_f):
            rgb[self.fast_idx] = self.rgb_f
            depth[self.fast_idx] = self.depth_f
        if len(self.ids_s):
            rgb[self.slow_idx] = self.rgb_s
            depth[self.slow_idx] = self.depth_s
        return rgb, depth
