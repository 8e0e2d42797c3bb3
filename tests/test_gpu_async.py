"""The render call is asynchronous and its device-detected errors are sticky.

gs_render_batch enqueues the whole render on the caller's stream and returns
without waiting for it (the C ABI's stated behaviour with sync_errors = 0); a
chunk that does not fit the workspace is reported by a later call, gs_sync or
gs_get_stats, after which rendering again succeeds. With sync_errors = 1 the
call waits and renders such a chunk again itself.
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


def test_render_returns_before_the_render_completes(torch):
    from paper_2510_15352_b300 import gs
    scene = synth.make_scene(300_000, 3, seed=3)
    W, H = 640, 480
    vm, it = synth.make_cameras(256, W, H, 480.0, (0.3, 1.2), seed=3)
    vm_d, it_d = torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda()
    stream = torch.cuda.current_stream()
    a = gs.Renderer(device=0, sync_errors=0)
    b = gs.Renderer(device=0, sync_errors=1)
    try:
        sa, sb = a.add_scene(scene), b.add_scene(scene)
        rgb_b, depth_b, _ = b.render(sb, vm_d, it_d, W, H, stream=stream)
        rgb_a, depth_a, _ = a.render(sa, vm_d, it_d, W, H, stream=stream)  # warm-up
        a.sync(stream)
        torch.cuda.synchronize()
        pending = []
        for _ in range(3):
            a.render(sa, vm_d, it_d, W, H, rgb_a, depth_a, stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
            pending.append(ev.query())  # False while the render still runs
        a.sync(stream)
        torch.cuda.synchronize()
        assert not all(pending), "every render had completed when its call returned"
        np.testing.assert_array_equal(rgb_a.cpu().numpy(), rgb_b.cpu().numpy())
        np.testing.assert_array_equal(depth_a.cpu().numpy(), depth_b.cpu().numpy())
    finally:
        a.close()
        b.close()


def _looking_away(torch, vm):
    """The same cameras turned to look straight up from high above the scene
    (almost nothing survives)."""
    up = torch.from_numpy(vm).cuda().clone()
    look_up = torch.tensor([[1.0, 0, 0], [0, 0, 1.0], [0, -1.0, 0]], device="cuda")
    up[:, :3, :3] = look_up
    up[:, :3, 3] = -(look_up @ torch.tensor([5.0, 5.0, 20.0], device="cuda"))
    return up


def test_overflow_is_reported_later_and_rendering_again_succeeds(torch, orc):
    """The first call of a batch size sizes the workspace (it waits); when the
    cameras then turn so that a chunk needs more, an asynchronous call cannot
    render it: the error comes with gs_sync (or gs_get_stats), once, and a
    render after it is complete and correct."""
    from paper_2510_15352_b300 import gs
    scene, vm, it, W, H = synth.workload("small_20k_8cam_160x120")
    vm_d, it_d = torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda()
    away = _looking_away(torch, vm)
    r = gs.Renderer(device=0, sync_errors=0, workspace_survivors=10)
    try:
        sid = r.add_scene(scene)
        r.render(sid, away, it_d, W, H)  # sizes the workspace for almost no survivors
        r.sync()
        r.render(sid, vm_d, it_d, W, H, want_T=True)  # returns: the overflow is on the device
        with pytest.raises(gs.GSError) as e:
            r.sync()
        assert e.value.status == gs.GS_ERR_CAPACITY
        r.sync()  # reported once
        rgb, depth, T = r.render(sid, vm_d, it_d, W, H, want_T=True)  # the workspace has grown
        r.sync()
        for c in (0, 5):
            ref = orc.render(scene, vm[c], it[c], W, H, bands=BANDS)
            res = compare_camera(rgb[c].cpu().numpy(), depth[c].cpu().numpy(),
                                 T[c].cpu().numpy(), ref)
            assert not res["unresolved"], res
        # the same error through gs_get_stats
        r2 = gs.Renderer(device=0, sync_errors=0, workspace_survivors=10)
        try:
            s2 = r2.add_scene(scene)
            r2.render(s2, away, it_d, W, H)
            r2.sync()
            r2.render(s2, vm_d, it_d, W, H)
            with pytest.raises(gs.GSError) as e:
                r2.stats()
            assert e.value.status == gs.GS_ERR_CAPACITY
        finally:
            r2.close()
    finally:
        r.close()
