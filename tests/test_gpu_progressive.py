"""The progressive depth order (gs_config.depth_prefix): the first phase orders
and bins each camera's nearest ranks only, tiles with live pixels at their
camera's cut save their state, and the second phase orders and bins the rest of
those cameras and resumes the tiles. Compositing visits every pixel's records in
the same order either way, so the images must be bit-identical to the whole
order's, and they must match the oracle."""
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
def gsmod(torch):
    from paper_2510_15352_b300 import gs
    return gs


def dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def render_all(torch, R, sid, vm, it, W, H):
    rgb, depth, T = R.render(sid, dev(torch, vm), dev(torch, it), W, H, want_T=True)
    R.sync()
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), depth.cpu().numpy(), T.cpu().numpy(), R.stats()


def test_default_prefix_is_progressive(gsmod):
    assert gsmod.default_config().depth_prefix == 0


@pytest.mark.parametrize("prefix", [1, 2049, 4096, 1_000_000])
def test_small_workload_second_phase_matches_oracle(torch, gsmod, orc, prefix):
    """The small workload (99 to 7,557 survivors per camera) with a cut after the
    first window (prefix 1), after two or four (for the camera of 4,125
    survivors the 4,096-rank cut falls inside its last bitmap word, so no word
    is left for the second phase although ranks are), or past every camera's
    survivors (no second phase): the images equal the whole order's bit for bit
    and match the oracle."""
    scene, vm, it, W, H = synth.workload("small_20k_8cam_160x120")
    R = gsmod.Renderer(device=0, depth_prefix=-1)
    try:
        sid = R.add_scene(scene)
        whole = render_all(torch, R, sid, vm, it, W, H)
        R.set_config(depth_prefix=prefix)
        part = render_all(torch, R, sid, vm, it, W, H)
        for a, b in zip(whole[:3], part[:3]):
            assert np.array_equal(a, b)
        st = part[3]
        if prefix < 1_000_000:  # (a camera whose tiles all stop before its cut has none)
            assert 1 <= st["depth_second_phase_cameras"] <= len(vm)
            assert st["depth_resumed_tiles"] > 0
        else:
            assert st["depth_second_phase_cameras"] == 0 and st["depth_resumed_tiles"] == 0
        assert whole[3]["depth_second_phase_cameras"] == 0
        for c in range(len(vm)):
            r = compare_camera(part[0][c], part[1][c], part[2][c],
                               orc.render(scene, vm[c], it[c], W, H, bands=BANDS))
            assert not r["unresolved"], (c, r)
    finally:
        R.close()


def test_full_size_chunk_equals_whole_order(torch, gsmod):
    """512 cameras of the full-size workload (1M Gaussians, 640x480, one chunk):
    the whole order, the default cut, a cut after the first window, and that cut
    with the saved-state list capped at 8 tiles (the rest are rendered again
    from rank 0) give the same images bit for bit. Before each render another
    512 cameras are rendered, so no workspace array still holds this batch's
    values from the render before."""
    scene, vm, it, W, H = synth.workload("single_1m_sh3_4096cam_640x480", n_cams=1024)
    R = gsmod.Renderer(device=0, depth_prefix=-1)
    try:
        sid = R.add_scene(scene)

        def run(**cfg):
            R.set_config(**cfg)
            render_all(torch, R, sid, vm[512:], it[512:], W, H)  # overwrite the workspace
            return render_all(torch, R, sid, vm[:512], it[:512], W, H)

        whole = run(depth_prefix=-1)
        default = run(depth_prefix=0)
        first = run(depth_prefix=1)
        R.set_resume_capacity(8)
        capped = run(depth_prefix=1)
        R.set_resume_capacity(0)
        for name, other in (("default", default), ("first", first), ("capped", capped)):
            for a, b in zip(whole[:3], other[:3]):
                assert np.array_equal(a, b), name
        sd, sf, sc = default[3], first[3], capped[3]
        print(f"\ncameras / tiles past their cut: default {sd['depth_second_phase_cameras']} / "
              f"{sd['depth_resumed_tiles']}, first window {sf['depth_second_phase_cameras']} / "
              f"{sf['depth_resumed_tiles']}")
        assert whole[3]["depth_second_phase_cameras"] == 0
        assert sf["depth_resumed_tiles"] > 8  # the capped run rendered some again
        assert sc["depth_resumed_tiles"] == sf["depth_resumed_tiles"]
        assert sf["depth_second_phase_cameras"] >= sd["depth_second_phase_cameras"]
        assert whole[3]["survivors"] == sd["survivors"] == sf["survivors"]
    finally:
        R.close()


def test_batched_scenes_equal_whole_order(torch, gsmod):
    """Five scenes of SH degree 2 with cameras at two resolutions in chunks of
    16: the records computed by the binning pass from each scene's rows (the
    progressive order, cut after the first window or by default) are those of
    the projection's write pass (the whole order), so the images are the same
    bit for bit."""
    scenes, which, vm, it, Ws, Hs = synth.make_batched(
        n_scenes=5, n_cams=40, seed=7, n_range=(5_000, 40_000), sh_degree=2,
        sizes=((128, 96, 100.0), (64, 48, 50.0)))
    vm_d, it_d = torch.from_numpy(vm).cuda(), torch.from_numpy(it).cuda()
    outs = {}
    for prefix in (-1, 0, 1):
        R = gsmod.Renderer(device=0, max_chunk_cameras=16, camera_group=8, depth_prefix=prefix)
        try:
            ids = np.array([R.add_scene(s) for s in scenes], dtype=np.int32)[which]
            rgb, depth, T, _ = R.render_v(ids, vm_d, it_d, Ws, Hs, want_T=True)
            R.sync()
            outs[prefix] = ([x.cpu().numpy() for x in (rgb, depth, T)], R.stats())
        finally:
            R.close()
    assert outs[1][1]["depth_second_phase_cameras"] > 0
    for p in (0, 1):
        for a, b in zip(outs[-1][0], outs[p][0]):
            assert np.array_equal(a, b), p
