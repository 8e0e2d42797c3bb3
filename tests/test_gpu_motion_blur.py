"""Motion blur (Sec. 3.3, Fig. 9): sub-frames offset along the camera velocity,
blended with equal weights; GPU against the FP64 oracle's blend of the same
sub-frames, and the degenerate cases (one sample, zero velocity)."""
from __future__ import annotations

import numpy as np
import pytest

from _parity import BANDS, TOL_DEPTH_REL, TOL_RGB
from paper_2510_15352_b300 import synth

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2510_15352_b300 import gs
    assert torch.cuda.is_available()
    scene = synth.make_scene(20_000, 2, seed=11)
    W, H = 160, 120
    vm, it = synth.make_cameras(4, W, H, 120.0, (0.3, 1.2), seed=11)
    vel = np.array([[1.5, 0.0, 0.0], [0.0, 2.0, 0.3], [-1.0, 1.0, 0.0], [0.0, 0.0, 0.0]],
                   dtype=np.float32)
    r = gs.Renderer(device=0)
    sid = r.add_scene(scene)
    yield torch, r, sid, scene, vm, it, vel, W, H
    r.close()


def test_motion_blur_matches_oracle_blend(setup, orc):
    torch, r, sid, scene, vm, it, vel, W, H = setup
    shutter, k = 0.06, 4
    rgb, depth, T = r.render_motion_blur(sid, torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda(),
                                         torch.from_numpy(vel).cuda(), shutter, k, W, H, want_T=True)
    torch.cuda.synchronize()
    rgb, depth, T = rgb.cpu().numpy(), depth.cpu().numpy(), T.cpu().numpy()
    for c in range(len(vm)):
        ref = O.render_motion_blur(orc, scene, vm[c], it[c], vel[c], shutter, k, W, H, bands=BANDS)
        e_rgb = np.abs(rgb[c] - ref["rgb"]).max(axis=-1)
        e_d = np.abs(depth[c] - ref["depth"])
        assert np.all(e_rgb <= TOL_RGB + ref["allow"]), e_rgb.max()
        assert np.all(e_d <= TOL_DEPTH_REL * np.maximum(np.abs(ref["depth"]), 1e-3) + ref["allow"])
        assert np.all(np.abs(T[c] - ref["T"]) <= TOL_RGB + ref["allow"])
    # a moving camera blurs: its blend differs from the sharp frame
    sharp, _, _ = r.render(sid, torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda(), W, H)
    torch.cuda.synchronize()
    assert np.abs(sharp.cpu().numpy()[0] - rgb[0]).max() > 0.05


def test_one_sample_and_zero_velocity_are_plain_renders(setup):
    torch, r, sid, scene, vm, it, vel, W, H = setup
    d_vm, d_it = torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda()
    plain, pd, _ = r.render(sid, d_vm, d_it, W, H)
    one, od, _ = r.render_motion_blur(sid, d_vm, d_it, torch.from_numpy(vel).cuda(), 0.1, 1, W, H)
    still, sd, _ = r.render_motion_blur(sid, d_vm, d_it, torch.zeros((4, 3), device="cuda"),
                                        0.1, 4, W, H)
    torch.cuda.synchronize()
    assert torch.equal(plain, one) and torch.equal(pd, od)
    np.testing.assert_allclose(still.cpu().numpy(), plain.cpu().numpy(), atol=1e-6)
