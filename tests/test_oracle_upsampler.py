"""Pins of the FP64 upsampler oracle against library routines, closed forms and
finite differences (CPU only)."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.signal
import torch

from oracle import upsampler as U


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 9, 3))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = U.conv3x3(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy.signal.correlate2d(x[n, :, :, c], W[o, c], mode="same")
                             for c in range(3))
            np.testing.assert_allclose(y[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_conv3x3_single_tap_is_a_shift():
    # a weight with one nonzero tap (u, v) moves the image by (u - 1, v - 1)
    x = np.arange(5 * 6, dtype=np.float64).reshape(1, 5, 6, 1)
    W = np.zeros((1, 1, 3, 3))
    W[0, 0, 2, 0] = 1.0
    y = U.conv3x3(x, W, np.zeros(1))[0, :, :, 0]
    ref = np.zeros((5, 6))
    ref[:4, 1:] = x[0, 1:, :5, 0]
    np.testing.assert_array_equal(y, ref)


def test_pixel_shuffle_brute_force_and_torch():
    rng = np.random.default_rng(1)
    z = rng.normal(size=(2, 3, 4, 48))
    o = U.pixel_shuffle(z)
    for n in range(2):
        for i in range(3):
            for j in range(4):
                for c in range(3):
                    for dy in range(4):
                        for dx in range(4):
                            assert o[n, 4 * i + dy, 4 * j + dx, c] == z[n, i, j, 16 * c + 4 * dy + dx]
    t = torch.nn.functional.pixel_shuffle(torch.from_numpy(z).permute(0, 3, 1, 2), 4)
    np.testing.assert_array_equal(o, t.permute(0, 2, 3, 1).numpy())
    np.testing.assert_array_equal(U.pixel_unshuffle(o), z)


def test_bilinear_matches_torch_and_reproduces_ramps():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 5, 7, 3))
    y = U.bilinear(x)
    t = torch.nn.functional.interpolate(torch.from_numpy(x).permute(0, 3, 1, 2), scale_factor=4,
                                        mode="bilinear", align_corners=False)
    np.testing.assert_allclose(y, t.permute(0, 2, 3, 1).numpy(), rtol=0, atol=1e-12)
    # a linear function of the pixel centre is reproduced exactly away from the
    # clamped border: LR centre k + 1/2 <-> HR centre 4k + 2
    h, w = 6, 8
    jj, ii = np.meshgrid(np.arange(w) + 0.5, np.arange(h) + 0.5)
    ramp = (0.3 * ii - 0.7 * jj + 1.0)[None, :, :, None]
    up = U.bilinear(ramp)[0, :, :, 0]
    JJ, II = np.meshgrid((np.arange(4 * w) + 0.5) / 4, (np.arange(4 * h) + 0.5) / 4)
    inner = (slice(2, 4 * h - 2), slice(2, 4 * w - 2))
    np.testing.assert_allclose(up[inner], (0.3 * II - 0.7 * JJ + 1.0)[inner], atol=1e-12)


def test_zero_last_layer_is_bilinear():
    rng = np.random.default_rng(3)
    rgb = rng.uniform(size=(1, 6, 5, 3))
    params = U.init_params(0, c_mid=8)
    np.testing.assert_allclose(U.forward(params, rgb), U.bilinear(rgb), atol=1e-15)


def test_box3_and_network_input():
    x = np.zeros((1, 4, 5, 3))
    x[0, 0, 0, 1] = 9.0          # corner: clamping counts it 4 times in its own mean
    x[0, 2, 2, 2] = 9.0          # interior
    b = U.box3(x)
    assert b[0, 0, 0, 1] == pytest.approx(4.0) and b[0, 1, 1, 1] == pytest.approx(1.0)
    assert b[0, 2, 2, 2] == pytest.approx(1.0) and b[0, 3, 3, 2] == pytest.approx(1.0)
    assert b[0, 0, 2, 2] == 0.0 and b[0, 3, 4, 0] == 0.0
    const = np.full((2, 3, 4, 3), 0.7)
    x0 = U.network_input(const)
    np.testing.assert_allclose(x0[..., :3], 0.2, atol=1e-15)
    np.testing.assert_allclose(x0[..., 3:], 0.0, atol=1e-14)
    x0 = U.network_input(x)
    np.testing.assert_allclose(x0[0, 2, 2, 5], U.DETAIL_SCALE * 8.0, rtol=1e-14)


def _fd_check(params, rgb, tgt, picks, h=1e-6):
    loss, grads = U.loss_and_grads(params, rgb, tgt)
    for li, kind, idx in picks:
        p = [(W.copy(), b.copy()) for W, b in params]
        arr = p[li][kind]
        a0 = arr[idx]
        arr[idx] = a0 + h
        lp = U.loss_and_grads(p, rgb, tgt)[0]
        arr[idx] = a0 - h
        lm = U.loss_and_grads(p, rgb, tgt)[0]
        fd = (lp - lm) / (2 * h)
        g = grads[li][kind][idx]
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)) + 1e-9, (li, kind, idx, fd, g)
    return loss


def test_gradients_match_central_differences():
    rng = np.random.default_rng(4)
    rgb = rng.uniform(size=(2, 5, 6, 3))
    tgt = rng.uniform(size=(2, 20, 24, 3))
    params = U.init_params(1, c_mid=6, zero_last=False)
    picks = []
    for li, (W, b) in enumerate(params):
        for _ in range(3):
            picks.append((li, 0, tuple(int(rng.integers(s)) for s in W.shape)))
        picks.append((li, 1, (int(rng.integers(b.shape[0])),)))
    _fd_check(params, rgb, tgt, picks)


def test_relu_gate_matters():
    # with a bias pushing layer 1 negative everywhere, every gradient below the
    # last layer vanishes; a dropped gate would leave them nonzero
    rng = np.random.default_rng(5)
    rgb = rng.uniform(size=(1, 4, 4, 3))
    tgt = rng.uniform(size=(1, 16, 16, 3))
    params = U.init_params(2, c_mid=4, zero_last=False)
    W0, b0 = params[0]
    params[0] = (W0 * 0.0, b0 - 1.0)
    _, grads = U.loss_and_grads(params, rgb, tgt)
    assert np.all(grads[0][0] == 0) and np.all(grads[1][0] == 0)
    assert np.any(grads[5][1] != 0)


def test_adam_first_step_closed_form():
    # bias-corrected first step: -lr * g / (|g| + eps) per element
    p = [(np.array([[[[1.0]]]]), np.array([2.0]))]
    g = [(np.array([[[[0.5]]]]), np.array([-3.0]))]
    opt = U.Adam(p, lr=0.1, eps=1e-8)
    q = opt.step(p, g)
    assert q[0][0].item() == pytest.approx(1.0 - 0.1 * 0.5 / (0.5 + 1e-8), abs=1e-15)
    assert q[0][1].item() == pytest.approx(2.0 + 0.1 * 3.0 / (3.0 + 1e-8), abs=1e-15)
    # second step with the same gradient moves by the same amount again
    r = opt.step(q, g)
    assert r[0][1].item() == pytest.approx(2.0 + 0.2 * 3.0 / (3.0 + 1e-8), abs=1e-12)


def test_psnr_definition():
    a = np.zeros((2, 2, 3))
    b = np.full((2, 2, 3), 0.1)
    assert U.psnr(a, b) == pytest.approx(20.0)
    assert U.psnr(a, a + 2.0) == pytest.approx(0.0)  # clamped to [0, 1]
