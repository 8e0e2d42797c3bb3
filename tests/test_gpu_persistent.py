"""The persistent binning + compositing launch (gs_config.persistent = 1).

One launch per chunk pulls binning items and then (camera, tile) compositing
items of every camera and scene of the chunk from a device queue; a tile waits
(bounded) for its camera's binning. Its images must equal those of the
separate binning and compositing launches bit for bit (the same arithmetic on
the same lists), in eager calls and in a captured CUDA graph; and a wait made
to run out must give GS_ERR_TIMEOUT without a fault or hang, after which the
context renders correctly.
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


def _batch():
    return synth.make_batched(n_scenes=5, n_cams=40, seed=7, n_range=(5_000, 40_000), sh_degree=2,
                              sizes=((128, 96, 100.0), (64, 48, 50.0)))


@pytest.mark.parametrize("comp_batch", [32, 64, 128])
def test_persistent_equals_separate_launches(torch, comp_batch):
    from paper_2510_15352_b300 import gs
    scenes, which, vm, it, Ws, Hs = _batch()
    vm_d, it_d = torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda()
    outs = []
    for persistent in (0, 1):
        r = gs.Renderer(device=0, persistent=persistent, comp_batch=comp_batch,
                        max_chunk_cameras=16, camera_group=8)
        try:
            ids = np.array([r.add_scene(s) for s in scenes], dtype=np.int32)[which]
            rgb, depth, T, _ = r.render_v(ids, vm_d, it_d, Ws, Hs, want_T=True)
            r.sync()
            outs.append([x.cpu().numpy() for x in (rgb, depth, T)])
            assert r.stats()["n_chunks"] == 3
        finally:
            r.close()
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


def test_persistent_full_resolution_against_oracle(torch, orc):
    from paper_2510_15352_b300 import gs
    scene = synth.make_scene(60_000, 3, seed=11)
    W, H = 640, 480
    vm, it = synth.make_cameras(6, W, H, 480.0, (0.3, 1.2), seed=11)
    r = gs.Renderer(device=0, persistent=1)
    try:
        sid = r.add_scene(scene)
        rgb, depth, T = r.render(sid, torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda(), W, H,
                                 want_T=True)
        r.sync()
        for c in (0, 5):
            ref = orc.render(scene, vm[c], it[c], W, H, bands=BANDS)
            res = compare_camera(rgb[c].cpu().numpy(), depth[c].cpu().numpy(), T[c].cpu().numpy(), ref)
            assert not res["unresolved"], res
    finally:
        r.close()


def test_persistent_launch_in_a_graph(torch):
    from paper_2510_15352_b300 import gs
    scenes, which, vm, it, Ws, Hs = _batch()
    vm_d, it_d = torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda()
    r = gs.Renderer(device=0, persistent=1, max_chunk_cameras=16, camera_group=8)
    try:
        ids = np.array([r.add_scene(s) for s in scenes], dtype=np.int32)[which]
        e_rgb, e_dep, e_T, _ = r.render_v(ids, vm_d, it_d, Ws, Hs, want_T=True)
        r.sync()
        P = int((Ws.astype(np.int64) * Hs).sum())
        rgb = torch.zeros((P, 3), device="cuda")
        dep = torch.zeros((P,), device="cuda")
        g = r.graph(ids, vm_d, it_d, Ws, Hs, rgb, dep)
        for _ in range(2):
            rgb.zero_()
            g.launch()
            g.check()
            assert torch.equal(rgb, e_rgb) and torch.equal(dep, e_dep)
        g.close()
    finally:
        r.close()


def test_bounded_wait_gives_up_and_the_context_recovers(torch, orc):
    from paper_2510_15352_b300 import gs
    scene, vm, it, W, H = synth.workload("small_20k_8cam_160x120")
    r = gs.Renderer(device=0, persistent=1)
    try:
        sid = r.add_scene(scene)
        vm0, it0 = torch.from_numpy(vm[:1]).cuda(), torch.from_numpy(it[:1]).cuda()
        assert r.timeout_probe(sid, vm0, it0, W, H) == gs.GS_ERR_TIMEOUT
        assert r.timeout_probe(sid, vm0, it0, W, H) == gs.GS_ERR_TIMEOUT  # again, same context
        r.sync()  # reported by the probe itself: nothing pending
        rgb, depth, T = r.render(sid, torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda(), W, H,
                                 want_T=True)
        r.sync()
        for c in (0, 7):
            ref = orc.render(scene, vm[c], it[c], W, H, bands=BANDS)
            res = compare_camera(rgb[c].cpu().numpy(), depth[c].cpu().numpy(), T[c].cpu().numpy(), ref)
            assert not res["unresolved"], res
    finally:
        r.close()
