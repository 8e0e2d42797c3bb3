"""CUDA-graph capture of a batched render (many scenes, mixed resolutions):
replays equal eager renders bit for bit, cameras updated in place are
honoured, a replay that outgrows the workspace is reported, and a workspace
reallocation invalidates the graph."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2510_15352_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def _setup(torch, gs, **cfg):
    scenes, which, vm, it, Ws, Hs = synth.make_batched(
        n_scenes=5, n_cams=40, seed=7, n_range=(5_000, 40_000), sh_degree=2,
        sizes=((128, 96, 100.0), (64, 48, 50.0)))
    r = gs.Renderer(device=0, max_chunk_cameras=16, camera_group=8, **cfg)
    ids = np.array([r.add_scene(s) for s in scenes], dtype=np.int32)[which]
    P = int((Ws.astype(np.int64) * Hs).sum())
    return r, ids, torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda(), Ws, Hs, P


def test_graph_replay_matches_eager(torch):
    from paper_2510_15352_b300 import gs
    r, ids, vm, it, Ws, Hs, P = _setup(torch, gs)
    try:
        rgb = torch.zeros((P, 3), device="cuda")
        dep = torch.zeros((P,), device="cuda")
        T = torch.zeros((P,), device="cuda")
        g = r.graph(ids, vm, it, Ws, Hs, rgb, dep, T)
        rgb.zero_(); dep.zero_(); T.zero_()
        g.launch()
        g.check()
        e_rgb, e_dep, e_T, _ = r.render_v(ids, vm, it, Ws, Hs, want_T=True)
        torch.cuda.synchronize()
        assert torch.equal(rgb, e_rgb) and torch.equal(dep, e_dep) and torch.equal(T, e_T)
        # cameras moved in place: the replay renders the new poses
        vm2 = torch.from_numpy(synth.make_batched(n_scenes=5, n_cams=40, seed=8,
                                                  n_range=(5_000, 40_000), sh_degree=2,
                                                  sizes=((128, 96, 100.0), (64, 48, 50.0)))[2]).cuda()
        vm.copy_(vm2)
        g.launch()
        g.check()
        e_rgb, e_dep, e_T, _ = r.render_v(ids, vm, it, Ws, Hs, want_T=True)
        torch.cuda.synchronize()
        assert torch.equal(rgb, e_rgb) and torch.equal(dep, e_dep) and torch.equal(T, e_T)
        assert float((T < 1).float().mean()) > 0.05
        g.close()
    finally:
        r.close()


def test_graph_overflow_and_invalidation(torch):
    from paper_2510_15352_b300 import gs
    # sync_errors = 1: the eager render below grows the workspace within the call
    r, ids, vm, it, Ws, Hs, P = _setup(torch, gs, workspace_survivors=1000, sync_errors=1)
    try:
        rgb = torch.zeros((P, 3), device="cuda")
        dep = torch.zeros((P,), device="cuda")
        # capture with every camera looking up, out of the scene: few survivors
        up = vm.clone()
        look_up = torch.tensor([[1.0, 0, 0], [0, 0, 1.0], [0, -1.0, 0]], device="cuda")
        up[:, :3, :3] = look_up
        up[:, :3, 3] = -(look_up @ torch.tensor([5.0, 5.0, 20.0], device="cuda"))
        cams = up.clone()
        g = r.graph(ids, cams, it, Ws, Hs, rgb, dep)
        cams.copy_(vm)  # now every camera sees its scene: far more survivors
        g.launch()
        with pytest.raises(gs.GSError) as e:
            g.check()
        assert e.value.status == gs.GS_ERR_CAPACITY
        # an eager render grows the workspace, which invalidates the graph
        r.render_v(ids, cams, it, Ws, Hs, rgb, dep)
        torch.cuda.synchronize()
        with pytest.raises(gs.GSError) as e:
            g.launch()
        assert e.value.status == gs.GS_ERR_INVALID_ARG
        g.close()
        g2 = r.graph(ids, cams, it, Ws, Hs, rgb, dep)
        g2.launch()
        g2.check()
        g2.close()
    finally:
        r.close()


def test_graph_invalidated_by_bitmap_growth(torch):
    """A render at twice the resolution grows the binning bitmaps (more
    super-tiles per camera) while the survivor buffers keep their size; the
    graph holds the old bitmap address, so launching it is refused."""
    from paper_2510_15352_b300 import gs
    r, ids, vm, it, Ws, Hs, P = _setup(torch, gs, workspace_survivors=4_000_000)
    try:
        rgb = torch.zeros((P, 3), device="cuda")
        dep = torch.zeros((P,), device="cuda")
        g = r.graph(ids, vm, it, Ws, Hs, rgb, dep)
        g.launch()
        g.check()
        W2, H2 = Ws * 2, Hs * 2
        r.render_v(ids, vm, it, W2, H2)
        torch.cuda.synchronize()
        with pytest.raises(gs.GSError) as e:
            g.launch()
        assert e.value.status == gs.GS_ERR_INVALID_ARG
        g.close()
    finally:
        r.close()
