"""The allocation-free segmented sort against the regular one.

gs_sort_segments_noalloc serves callers that cannot allocate GPU memory (its
scratch is a fixed device array inside the library). It must give exactly the
result of gs_sort_segments -- integer keys, so the tolerance is zero -- and keep
doing so on a second call in a row, which reuses the same scratch. This file
is collected last so a run that stops at its first failure has run every
other test first; it also passes alone in a fresh process.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _case(seed):
    rng = np.random.default_rng(seed)
    lens = [0, 1, 33, 2048, 2049, 5000, 70_001, 3, 12_345]
    starts, pos = [], 0
    for L in lens:
        pos += int(rng.integers(0, 4))
        starts.append(pos)
        pos += L
    n = pos + 2
    keys = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    keys[::5] = keys[1]  # ties, so stability matters
    vals = (np.arange(n, dtype=np.uint32) * np.uint32(2654435761)) & np.uint32(0xFFFFFFFF)
    return keys, vals, np.array(starts, np.int64), np.array(lens, np.int64)


def test_noalloc_sort_matches_regular_sort_twice():
    import torch
    from paper_2510_15352_b300 import gs
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    r = gs.Renderer(device=0)
    try:
        for seed in (0, 1):  # two calls in a row share the library's scratch
            keys, vals, ss, sc = _case(seed)
            a_k = torch.from_numpy(keys.view(np.int32).copy()).cuda()
            a_v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
            b_k, b_v = a_k.clone(), a_v.clone()
            d_s = torch.from_numpy(ss).cuda()
            d_c = torch.from_numpy(sc).cuda()
            r.sort_segments(a_k, a_v, d_s, d_c)
            stream = torch.cuda.current_stream().cuda_stream or None
            st = gs.gs_sort_segments_noalloc(b_k.data_ptr(), b_v.data_ptr(), b_k.numel(),
                                             d_s.data_ptr(), d_c.data_ptr(), len(ss), stream)
            assert st == gs.GS_OK
            torch.cuda.synchronize()
            np.testing.assert_array_equal(b_k.cpu().numpy(), a_k.cpu().numpy())
            np.testing.assert_array_equal(b_v.cpu().numpy(), a_v.cpu().numpy())
            # and the regular sort is the stable argsort
            o = np.argsort(keys[ss[5]:ss[5] + sc[5]], kind="stable")
            np.testing.assert_array_equal(a_k.cpu().numpy().view(np.uint32)[ss[5]:ss[5] + sc[5]],
                                          keys[ss[5]:ss[5] + sc[5]][o])
    finally:
        r.close()


def _run_noalloc(gs, torch, k, v, ss, sc):
    d_s = torch.from_numpy(ss).cuda()
    d_c = torch.from_numpy(sc).cuda()
    stream = torch.cuda.current_stream().cuda_stream or None
    st = gs.gs_sort_segments_noalloc(k.data_ptr(), v.data_ptr(), k.numel(), d_s.data_ptr(),
                                     d_c.data_ptr(), len(ss), stream)
    torch.cuda.synchronize()
    return st


def test_noalloc_sort_at_its_limits():
    """2,097,152 keys in 4,096 segments (both limits; the scratch's every region
    in use): bit for bit the regular sort's result."""
    import torch
    from paper_2510_15352_b300 import gs
    rng = np.random.default_rng(7)
    n, n_seg = 1 << 21, 4096
    cuts = np.sort(rng.integers(0, n + 1, size=n_seg - 1))
    bounds = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    ss, sc = bounds[:-1].copy(), np.diff(bounds).astype(np.int64)
    sc[5] = 0  # an empty segment among them
    keys = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    keys[::7] = keys[3]
    vals = np.arange(n, dtype=np.uint32)
    r = gs.Renderer(device=0)
    try:
        a_k = torch.from_numpy(keys.view(np.int32).copy()).cuda()
        a_v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
        b_k, b_v = a_k.clone(), a_v.clone()
        r.sort_segments(a_k, a_v, torch.from_numpy(ss).cuda(), torch.from_numpy(sc).cuda())
        assert _run_noalloc(gs, torch, b_k, b_v, ss, sc) == gs.GS_OK
        np.testing.assert_array_equal(b_k.cpu().numpy(), a_k.cpu().numpy())
        np.testing.assert_array_equal(b_v.cpu().numpy(), a_v.cpu().numpy())
    finally:
        r.close()


def test_noalloc_sort_out_of_range_segment_is_empty():
    """A segment reaching past n is treated as empty (its keys stay as they
    are) while the other segments still sort."""
    import torch
    from paper_2510_15352_b300 import gs
    rng = np.random.default_rng(8)
    n = 5000
    keys = rng.integers(0, 1000, size=n, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    ss = np.array([0, 1000, 4995], np.int64)
    sc = np.array([1000, 3000, 10], np.int64)  # the last one ends at 5005 > n
    k = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    assert _run_noalloc(gs, torch, k, v, ss, sc) == gs.GS_OK
    gk, gv = k.cpu().numpy().view(np.uint32), v.cpu().numpy().view(np.uint32)
    for s0, c0 in ((0, 1000), (1000, 3000)):
        o = np.argsort(keys[s0:s0 + c0], kind="stable")
        np.testing.assert_array_equal(gk[s0:s0 + c0], keys[s0:s0 + c0][o])
        np.testing.assert_array_equal(gv[s0:s0 + c0], vals[s0:s0 + c0][o])
    np.testing.assert_array_equal(gk[4000:], keys[4000:])
    np.testing.assert_array_equal(gv[4000:], vals[4000:])


def test_noalloc_sort_rejects_oversize_requests():
    from paper_2510_15352_b300 import gs
    p = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert gs.gs_sort_segments_noalloc(p, p, (1 << 21) + 1, p, p, 1, None) == gs.GS_ERR_CAPACITY
    assert gs.gs_sort_segments_noalloc(p, p, 10, p, p, 4097, None) == gs.GS_ERR_CAPACITY
