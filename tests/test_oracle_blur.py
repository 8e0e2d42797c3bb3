"""Pins of the oracle's motion blur (Sec. 3.3 and Fig. 9: a few frames offset
along the camera's velocity, alpha-blended).

Reading pinned here: k sub-frames in time order span the shutter interval
centred on the given pose, the camera keeps its orientation and its centre
moves along the velocity, and the sub-frames are blended with equal weights.
The pins do not restate that formula: they check geometric facts of the
poses (each pose's camera centre recovered by inverting it, equal spacing,
symmetry about the given centre, span = velocity x shutter), the closed-form
image of one Gaussian seen from every sub-frame (projection of a point offset
along x, with the off-axis EWA Jacobian written out by hand), and the blend's
weights (identical sub-frames blend to the single frame). Planted mistakes in
copies of the two functions (sign of the offset, offsets j/k - 1/2, transposed
rotation, weights not summing to one, a dropped sub-frame) must each fail a pin.
"""
from __future__ import annotations

import inspect
import math
import types

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from _cases import Y00, dc_for_colour, f32, identity_camera, logit, scene_from

import oracle as O


def _centre(V):
    """Camera centre of a world->camera pose: the point mapped to the origin."""
    V = np.asarray(V, dtype=np.float64)
    return np.linalg.solve(V[:3, :3], -V[:3, 3])


def _random_pose(rng):
    R = Rotation.from_quat(rng.normal(size=4)).as_matrix()
    C = rng.uniform(-3, 3, size=3)
    V = np.eye(4)
    V[:3, :3] = R
    V[:3, 3] = -R @ C
    return V, C


def pin_pose_geometry(blur_poses, render_motion_blur, orc):
    rng = np.random.default_rng(11)
    for k in (2, 3, 4, 7):
        V, C = _random_pose(rng)
        v = rng.normal(size=3)
        s = rng.uniform(0.02, 0.5)
        P = blur_poses(V, v, s, k)
        assert len(P) == k
        cs = np.array([_centre(p) for p in P])
        for p in P:  # orientation kept, still a rigid pose
            np.testing.assert_allclose(p[:3, :3], V[:3, :3], atol=1e-14)
            np.testing.assert_allclose(p[3], [0, 0, 0, 1], atol=0)
        steps = np.diff(cs, axis=0)
        for d in steps:  # equally spaced along the velocity
            np.testing.assert_allclose(d, steps[0], atol=1e-12)
        np.testing.assert_allclose(cs[-1] - cs[0], v * s, atol=1e-12)  # time order, span v s
        np.testing.assert_allclose(cs.mean(axis=0), C, atol=1e-12)  # centred on the pose


def pin_degenerate_poses(blur_poses, render_motion_blur, orc):
    rng = np.random.default_rng(12)
    V, _ = _random_pose(rng)
    v = rng.normal(size=3)
    (only,) = blur_poses(V, v, 0.3, 1)  # one sample: the pose itself
    np.testing.assert_allclose(only, V, atol=1e-14)
    for p in blur_poses(V, v, 0.0, 5):  # zero shutter time
        np.testing.assert_allclose(p, V, atol=1e-14)
    for p in blur_poses(V, np.zeros(3), 0.2, 4):  # at rest
        np.testing.assert_allclose(p, V, atol=1e-14)


def _image_of_point_gaussian(W, H, f, x, z, s, o, col):
    """Closed-form render of one isotropic Gaussian (scale s) whose mean is at
    camera coordinates (x, 0, z) with an identity camera rotation. The EWA
    Jacobian at (x, 0, z) is [[f/z, 0, -f x/z^2], [0, f/z, 0]], so the 2D
    covariance is diag((f s/z)^2 (1 + x^2/z^2) + 0.3, (f s/z)^2 + 0.3); the
    image centre is (W/2 + f x/z, H/2). Tile rect from the 3-sigma radius."""
    a = (f * s / z) ** 2 * (1 + (x / z) ** 2) + 0.3
    c = (f * s / z) ** 2 + 0.3
    u0, v0 = W / 2 + f * x / z, H / 2
    r = 3 * math.sqrt(max(a, c))
    TX, TY = (W + 15) // 16, (H + 15) // 16
    rect = [max(0, math.floor((u0 - r) / 16)), min(TX - 1, math.floor((u0 + r) / 16)),
            max(0, math.floor((v0 - r) / 16)), min(TY - 1, math.floor((v0 + r) / 16))]
    jj, ii = np.mgrid[0:H, 0:W]
    dx, dy = ii + 0.5 - u0, jj + 0.5 - v0
    al = np.minimum(0.99, o * np.exp(-0.5 * (dx * dx / a + dy * dy / c)))
    tx, ty = ii // 16, jj // 16
    inrect = (tx >= rect[0]) & (tx <= rect[1]) & (ty >= rect[2]) & (ty <= rect[3])
    al = np.where((al >= 1 / 255) & inrect, al, 0.0)
    cols = 0.5 + Y00 * np.array([f32(c_) for c_ in dc_for_colour(col)])
    return al[..., None] * cols, al * z, 1 - al


_W, _H, _F = 64, 48, 60.0
_Z, _S, _O, _COL = 2.0, 0.08, 0.8, (0.9, 0.3, 0.2)


def _one_gaussian():
    return scene_from([[0.0, 0.0, _Z]], [math.log(_S)] * 3, [1, 0, 0, 0], logit(_O), colours=_COL)


def _rounded():
    return f32(_Z), math.exp(f32(math.log(_S))), 1 / (1 + math.exp(-f32(logit(_O))))


def _pin_subframes_closed_form(blur_poses, render_motion_blur, orc, k):
    # identity camera moving along +x at 2 m/s, shutter 0.1 s: sub-frame j has
    # its centre at x_j = 0.2 (j/(k-1) - 1/2), so the Gaussian at world x = 0
    # sits at camera x = -x_j
    sc = _one_gaussian()
    vm, it = identity_camera(_W, _H, _F)
    v, s = np.array([2.0, 0.0, 0.0]), 0.1
    z, ss, o = _rounded()
    P = blur_poses(vm, v, s, k)
    xs = [-v[0] * s * (j / (k - 1) - 0.5) for j in range(k)]
    for j, Vj in enumerate(P):
        out = orc.render(sc, Vj, it, _W, _H)
        rgb, dep, T = _image_of_point_gaussian(_W, _H, _F, xs[j], z, ss, o, _COL)
        np.testing.assert_allclose(out["rgb"], rgb, atol=1e-12)
        np.testing.assert_allclose(out["depth"], dep, atol=1e-12)
        np.testing.assert_allclose(out["T"], T, atol=1e-12)
    # the first sub-frame (camera furthest back, at -x) sees the Gaussian right of centre
    assert _centre(P[0])[0] < 0


def pin_subframes_closed_form(blur_poses, render_motion_blur, orc):
    for k in (2, 3, 4):
        _pin_subframes_closed_form(blur_poses, render_motion_blur, orc, k)


def pin_blend_closed_form(blur_poses, render_motion_blur, orc):
    sc = _one_gaussian()
    vm, it = identity_camera(_W, _H, _F)
    v, s, k = np.array([2.0, 0.0, 0.0]), 0.1, 3
    z, ss, o = _rounded()
    got = render_motion_blur(orc, sc, vm, it, v, s, k, _W, _H)
    parts = [_image_of_point_gaussian(_W, _H, _F, -v[0] * s * (j / (k - 1) - 0.5), z, ss, o, _COL)
             for j in range(k)]
    np.testing.assert_allclose(got["rgb"], sum(p[0] for p in parts) / k, atol=1e-12)
    np.testing.assert_allclose(got["depth"], sum(p[1] for p in parts) / k, atol=1e-12)
    np.testing.assert_allclose(got["T"], sum(p[2] for p in parts) / k, atol=1e-12)
    assert np.all(got["allow"] == 0)  # no decision near a threshold in this scene


def pin_blend_weights(blur_poses, render_motion_blur, orc):
    # a camera at rest: every sub-frame is the same frame, so equal weights that
    # sum to one give back the plain render (exactly up to rounding)
    sc = _one_gaussian()
    vm, it = identity_camera(_W, _H, _F)
    plain = orc.render(sc, vm, it, _W, _H)
    for k in (1, 2, 5):
        got = render_motion_blur(orc, sc, vm, it, np.zeros(3), 0.1, k, _W, _H)
        for key in ("rgb", "depth", "T"):
            np.testing.assert_allclose(got[key], plain[key], atol=1e-14, rtol=0)
    # and the blend is linear: T + sum of weights stays 1 per pixel through the blend
    got = render_motion_blur(orc, sc, vm, it, np.array([0.0, 1.5, 0.0]), 0.1, 4, _W, _H)
    z, _, _ = _rounded()
    np.testing.assert_allclose(got["depth"] / z + got["T"], 1.0, atol=1e-12)


PINS = [pin_pose_geometry, pin_degenerate_poses, pin_subframes_closed_form,
        pin_blend_closed_form, pin_blend_weights]


@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_blur_pin(pin, orc):
    pin(O.blur_poses, O.render_motion_blur, orc)


# ----------------------------------------------------------------- mutants

MUTANTS = {
    "offset_sign": ("W[:3, 3] = t - R @ (v * shutter * frac)",
                    "W[:3, 3] = t + R @ (v * shutter * frac)"),
    "offset_j_over_k": ("frac = j / (samples - 1) - 0.5", "frac = j / samples - 0.5"),
    "offset_not_centred": ("frac = j / (samples - 1) - 0.5", "frac = j / (samples - 1)"),
    "rotation_transposed": ("W[:3, 3] = t - R @ (v * shutter * frac)",
                            "W[:3, 3] = t - R.T @ (v * shutter * frac)"),
    "no_rotation": ("W[:3, 3] = t - R @ (v * shutter * frac)",
                    "W[:3, 3] = t - (v * shutter * frac)"),
    "weights_not_normalised": ("acc[k] = acc[k] + part[k] / samples",
                               "acc[k] = acc[k] + part[k] / (samples + 1)"),
    "last_subframe_dropped": ("for V in blur_poses(viewmat, velocity, shutter, samples):",
                              "for V in blur_poses(viewmat, velocity, shutter, samples)[:-1]:"),
}


def _mutated(name):
    """Copies of blur_poses and render_motion_blur with one planted mistake,
    compiled from the oracle's own source text."""
    old, new = MUTANTS[name]
    ns = {"np": np, "Oracle": O.Oracle, "_f64": O._f64}
    src = ""
    for fn in (O.blur_poses, O.render_motion_blur):
        src += inspect.getsource(fn) + "\n"
    assert src.count(old) == 1, f"mutant anchor for {name} not unique"
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), ns)
    return types.SimpleNamespace(blur_poses=ns["blur_poses"],
                                 render_motion_blur=ns["render_motion_blur"])


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_blur_mutant_is_caught(name, orc):
    m = _mutated(name)
    # render_motion_blur looks blur_poses up in its own namespace: the mutant's
    caught = []
    for pin in PINS:
        try:
            pin(m.blur_poses, m.render_motion_blur, orc)
        except Exception:  # a failed assertion, or a pin that cannot even run
            caught.append(pin.__name__)
    assert caught, f"planted mistake {name!r} passed every motion-blur pin"


def test_unmutated_copy_passes_every_pin(orc):
    ns = {"np": np, "Oracle": O.Oracle, "_f64": O._f64}
    src = inspect.getsource(O.blur_poses) + "\n" + inspect.getsource(O.render_motion_blur)
    exec(compile(src, "<copy>", "exec"), ns)
    for pin in PINS:
        pin(ns["blur_poses"], ns["render_motion_blur"], orc)
