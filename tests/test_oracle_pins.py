"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something it does not compute itself:
closed forms of special cases, textbook spherical harmonics written out in
Cartesian form, quadrature, library rotations, rigid-motion invariance,
the telescoping identity sum_i w_i + T = 1, and brute force. The method is
the 3DGS rasteriser the paper uses as its renderer (Sec. 3.2; depth as a
by-product, Fig. 4).
"""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from _cases import Y00, dc_for_colour, f32, identity_camera, logit, scene_from

import oracle as O

# ------------------------------------------------------------------ SH basis


def cartesian_sh(x, y, z):
    """Real SH with the Condon-Shortley phase, l <= 3, in Cartesian form
    (textbook table; constants as closed-form square roots)."""
    s = math.sqrt
    pi = math.pi
    return np.array([
        1.0 / (2.0 * s(pi)),
        -s(3 / (4 * pi)) * y, s(3 / (4 * pi)) * z, -s(3 / (4 * pi)) * x,
        s(15 / (4 * pi)) * x * y, -s(15 / (4 * pi)) * y * z, s(5 / (16 * pi)) * (3 * z * z - 1),
        -s(15 / (4 * pi)) * x * z, s(15 / (16 * pi)) * (x * x - y * y),
        -s(35 / (32 * pi)) * y * (3 * x * x - y * y), s(105 / (4 * pi)) * x * y * z,
        -s(21 / (32 * pi)) * y * (5 * z * z - 1), s(7 / (16 * pi)) * z * (5 * z * z - 3),
        -s(21 / (32 * pi)) * x * (5 * z * z - 1), s(105 / (16 * pi)) * z * (x * x - y * y),
        -s(35 / (32 * pi)) * x * (x * x - 3 * y * y),
    ])


def test_sh_matches_cartesian_table(orc):
    rng = np.random.default_rng(5)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d[0] = [0, 0, 1]
    d[1] = [0, 0, -1]
    d[2] = [1, 0, 0]
    got = orc.sh_basis(3, d)
    want = np.stack([cartesian_sh(*v) for v in d])
    np.testing.assert_allclose(got, want, atol=1e-13, rtol=0)
    # lower degrees are prefixes
    np.testing.assert_allclose(orc.sh_basis(1, d), want[:, :4], atol=1e-13)


def test_sh_orthonormal_by_quadrature(orc):
    xs, ws = np.polynomial.legendre.leggauss(12)  # exact for degree <= 23 in cos(theta)
    nphi = 16
    phis = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    dirs, wts = [], []
    for ct, w in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            dirs.append([st * math.cos(ph), st * math.sin(ph), ct])
            wts.append(w * 2 * math.pi / nphi)
    Y = orc.sh_basis(3, np.array(dirs))
    G = (Y * np.array(wts)[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


# ------------------------------------------------------------- geometry


def test_quaternion_rotation_matches_library(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = rng.normal(size=4) * rng.uniform(0.1, 5)  # unnormalised on purpose
        R = orc.quat_to_rot(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: (x,y,z,w)
        np.testing.assert_allclose(R, ref, atol=1e-13)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(R) - 1) < 1e-12
    th = 0.7
    Rz = orc.quat_to_rot([math.cos(th / 2), 0, 0, math.sin(th / 2)])
    np.testing.assert_allclose(Rz, [[math.cos(th), -math.sin(th), 0],
                                    [math.sin(th), math.cos(th), 0], [0, 0, 1]], atol=1e-15)


def test_cov3d_is_rotated_diag(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        ls = rng.normal(-2, 1, size=3)
        q = rng.normal(size=4)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        want = R @ np.diag(np.exp(2 * ls)) @ R.T
        np.testing.assert_allclose(orc.cov3d(ls, q), want, rtol=1e-12, atol=1e-16)


# --------------------------------------------------- single Gaussian, closed form


@pytest.mark.parametrize("z,s,o,col", [(2.0, 0.05, 0.7, (0.9, 0.4, 0.1)),
                                       (5.0, 0.2, 0.95, (0.2, 0.8, 0.5)),
                                       (0.8, 0.01, 0.3, (1.0, 1.0, 1.0))])
def test_single_gaussian_closed_form(orc, z, s, o, col):
    W, H, f = 64, 48, 60.0
    sc = scene_from([[0.0, 0.0, z]], [math.log(s)] * 3, [1, 0, 0, 0], logit(o), colours=col)
    vm, it = identity_camera(W, H, f)
    zz, ss, oo = f32(z), math.exp(f32(math.log(s))), 1 / (1 + math.exp(-f32(logit(o))))
    sig2 = (f * ss / zz) ** 2 + 0.3
    cols = 0.5 + Y00 * np.array([f32(v) for v in dc_for_colour(col)])
    rec = orc.project(sc, vm, it, W, H)
    assert rec["valid"][0]
    np.testing.assert_allclose([rec["u"][0], rec["v"][0]], [W / 2, H / 2], atol=1e-12)
    np.testing.assert_allclose([rec["A"][0], rec["B"][0], rec["C"][0]], [1 / sig2, 0, 1 / sig2],
                               rtol=1e-12, atol=1e-15)
    r = 3 * math.sqrt(sig2)
    np.testing.assert_allclose(rec["r"][0], r, rtol=1e-12)
    TX, TY = (W + 15) // 16, (H + 15) // 16
    want_rect = [max(0, math.floor((W / 2 - r) / 16)), min(TX - 1, math.floor((W / 2 + r) / 16)),
                 max(0, math.floor((H / 2 - r) / 16)), min(TY - 1, math.floor((H / 2 + r) / 16))]
    assert list(rec["rect"][0]) == want_rect
    out = orc.render(sc, vm, it, W, H)
    jj, ii = np.mgrid[0:H, 0:W]
    d2 = (ii + 0.5 - W / 2) ** 2 + (jj + 0.5 - H / 2) ** 2
    a = np.minimum(0.99, oo * np.exp(-d2 / (2 * sig2)))
    tx, ty = ii // 16, jj // 16
    inrect = (tx >= want_rect[0]) & (tx <= want_rect[1]) & (ty >= want_rect[2]) & (ty <= want_rect[3])
    a = np.where((a >= 1 / 255) & inrect, a, 0.0)
    np.testing.assert_allclose(out["rgb"], a[..., None] * cols, atol=1e-12)
    np.testing.assert_allclose(out["depth"], a * zz, atol=1e-12)
    np.testing.assert_allclose(out["T"], 1 - a, atol=1e-12)


def test_sheared_footprint_pixels(orc):
    """A Gaussian turned about the optical axis, with fx != fy: its footprint
    is diag(fx, fy)/z * Sigma_xy * diag(fx, fy)/z + 0.3 I, and every pixel is
    o * exp(-d^T inv(Sigma') d / 2), inverted here with a library inverse."""
    W, H, fx, fy, z = 64, 64, 70.0, 45.0, 2.0
    th = 0.6
    s = (0.15, 0.04, 0.05)
    sc = scene_from([[0.0, 0.0, z]], np.log(s), [math.cos(th / 2), 0, 0, math.sin(th / 2)],
                    logit(0.9), colours=(1.0, 1.0, 1.0))
    vm, it = identity_camera(W, H, fx, fy)
    q = [f32(math.cos(th / 2)), 0.0, 0.0, f32(math.sin(th / 2))]
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    sig = R @ np.diag([math.exp(2 * f32(math.log(v))) for v in s]) @ R.T
    Jd = np.diag([fx / f32(z), fy / f32(z)])
    cov = Jd @ sig[:2, :2] @ Jd + 0.3 * np.eye(2)
    inv = np.linalg.inv(cov)
    assert abs(inv[0, 1]) > 1e-3  # really sheared
    o = 1 / (1 + math.exp(-f32(logit(0.9))))
    col = 0.5 + Y00 * f32(dc_for_colour(1.0))
    out = orc.render(sc, vm, it, W, H)
    r = 3 * math.sqrt(np.linalg.eigvalsh(cov).max())
    jj, ii = np.mgrid[0:H, 0:W]
    dx, dy = ii + 0.5 - W / 2, jj + 0.5 - H / 2
    a = np.minimum(0.99, o * np.exp(-0.5 * (inv[0, 0] * dx * dx + 2 * inv[0, 1] * dx * dy +
                                            inv[1, 1] * dy * dy)))
    tx, ty = ii // 16, jj // 16
    inrect = ((tx >= math.floor((W / 2 - r) / 16)) & (tx <= math.floor((W / 2 + r) / 16)) &
              (ty >= math.floor((H / 2 - r) / 16)) & (ty <= math.floor((H / 2 + r) / 16)))
    a = np.where((a >= 1 / 255) & inrect, a, 0.0)
    np.testing.assert_allclose(out["rgb"][..., 0], a * col, atol=1e-12)


@pytest.mark.parametrize("fx,fy", [(50.0, 50.0), (50.0, 35.0)])
def test_off_axis_anisotropic_jacobian(orc, fx, fy):
    """Axis-aligned Gaussian off the optical axis: Sigma' from J by hand."""
    W, H = 80, 60
    p = (0.3, -0.2, 2.0)
    s = (0.05, 0.02, 0.08)
    sc = scene_from([p], np.log(s), [1, 0, 0, 0], 0.0)
    vm, it = identity_camera(W, H, fx, fy)
    x, y, z = (f32(v) for v in p)
    s1, s2, s3 = (math.exp(f32(math.log(v))) for v in s)
    a = (fx / z) ** 2 * s1 ** 2 + (fx * x / z ** 2) ** 2 * s3 ** 2 + 0.3
    b = (fx * x / z ** 2) * (fy * y / z ** 2) * s3 ** 2
    c = (fy / z) ** 2 * s2 ** 2 + (fy * y / z ** 2) ** 2 * s3 ** 2 + 0.3
    rec = orc.project(sc, vm, it, W, H)
    np.testing.assert_allclose([rec["a"][0], rec["b"][0], rec["c"][0]], [a, b, c], rtol=1e-12)
    np.testing.assert_allclose([rec["u"][0], rec["v"][0]], [fx * x / z + W / 2, fy * y / z + H / 2],
                               rtol=1e-13)
    det = a * c - b * b
    np.testing.assert_allclose([rec["A"][0], rec["B"][0], rec["C"][0]], [c / det, -b / det, a / det],
                               rtol=1e-12)
    lam = 0.5 * (a + c) + math.sqrt(0.25 * (a - c) ** 2 + b * b)
    np.testing.assert_allclose(rec["r"][0], 3 * math.sqrt(lam), rtol=1e-12)


def test_guard_band_clamp(orc):
    """Far off-screen Gaussian: J uses x/z clamped to 1.3 * (W/2) / fx."""
    W, H, f = 80, 60, 50.0
    p = (3.0, 0.1, 2.0)  # x/z = 1.5 > 1.3 * 40 / 50 = 1.04
    s = (0.3, 0.3, 0.3)
    sc = scene_from([p], np.log(s), [1, 0, 0, 0], 0.0)
    vm, it = identity_camera(W, H, f)
    x, y, z = (f32(v) for v in p)
    ss = math.exp(f32(math.log(0.3)))
    lim = 1.3 * (W / 2) / f
    xt = lim * z
    a = (f / z) ** 2 * ss ** 2 + (f * xt / z ** 2) ** 2 * ss ** 2 + 0.3
    b = (f * xt / z ** 2) * (f * y / z ** 2) * ss ** 2
    rec = orc.project(sc, vm, it, W, H)
    np.testing.assert_allclose([rec["a"][0], rec["b"][0]], [a, b], rtol=1e-12)


# --------------------------------------------------------- ordering, stopping


def test_two_gaussians_depth_order(orc):
    W, H, f = 32, 32, 40.0
    c1, c2 = (1.0, 0.0, 0.0), (0.0, 0.0, 1.0)
    o1, o2 = 0.6, 0.8
    vm, it = identity_camera(W, H, f)
    px = (W // 2, H // 2)

    def render(z1, z2):
        sc = scene_from([[0, 0, z1], [0, 0, z2]], [math.log(0.05)] * 3, [1, 0, 0, 0],
                        [logit(o1), logit(o2)], colours=[c1, c2])
        out = orc.render(sc, vm, it, W, H)
        rec = orc.project(sc, vm, it, W, H)
        return out, rec

    out, rec = render(2.0, 3.0)
    j, i = px[1], px[0]
    d2 = lambda k: (i + 0.5 - rec["u"][k]) ** 2 + (j + 0.5 - rec["v"][k]) ** 2
    a1 = rec["o"][0] * math.exp(-0.5 * rec["A"][0] * d2(0))
    a2 = rec["o"][1] * math.exp(-0.5 * rec["A"][1] * d2(1))
    col = lambda k: np.array([rec["red"][k], rec["green"][k], rec["blue"][k]])
    np.testing.assert_allclose(out["rgb"][j, i], a1 * col(0) + (1 - a1) * a2 * col(1), atol=1e-12)
    np.testing.assert_allclose(out["depth"][j, i], a1 * rec["z"][0] + (1 - a1) * a2 * rec["z"][1],
                               atol=1e-12)
    # swapped depths: the second Gaussian is in front now
    out2, rec2 = render(3.0, 2.0)
    a1 = rec2["o"][0] * math.exp(-0.5 * rec2["A"][0] * d2(0))
    a2 = rec2["o"][1] * math.exp(-0.5 * rec2["A"][1] * d2(1))
    np.testing.assert_allclose(out2["rgb"][j, i], a2 * col(1) + (1 - a2) * a1 * col(0), atol=1e-12)
    # equal depths: index order decides (Gaussian 0 first)
    out3, rec3 = render(2.5, 2.5)
    a1 = rec3["o"][0] * math.exp(-0.5 * rec3["A"][0] * d2(0))
    a2 = rec3["o"][1] * math.exp(-0.5 * rec3["A"][1] * d2(1))
    np.testing.assert_allclose(out3["rgb"][j, i], a1 * col(0) + (1 - a1) * a2 * col(1), atol=1e-12)


def test_termination_excludes_crossing_gaussian(orc):
    """alpha = 0.99 (clamped) at the centre: T goes 1 -> 0.01 -> 1e-4 (kept,
    not < 1e-4) -> 1e-6 (< 1e-4: the third one stops the walk, not added)."""
    W, H, f = 16, 16, 20.0
    cols = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]
    sc = scene_from([[0, 0, 1.0 + k] for k in range(4)], [math.log(2.0)] * 3, [1, 0, 0, 0],
                    logit(0.9999), colours=cols)
    vm, it = identity_camera(W, H, f)
    out = orc.render(sc, vm, it, W, H)
    rec = orc.project(sc, vm, it, W, H)
    j = i = 8
    # the pixel centre is 0.5 px off the mean; alpha is still clamped at 0.99
    alphas = [min(0.99, rec["o"][k] * math.exp(-0.5 * rec["A"][k] * 0.5)) for k in range(4)]
    assert all(a == 0.99 for a in alphas)
    T1 = 1 - 0.99
    T2 = T1 * (1 - 0.99)
    assert T2 >= 1e-4 and T2 * (1 - 0.99) < 1e-4
    col = lambda k: np.array([rec["red"][k], rec["green"][k], rec["blue"][k]])
    want = 0.99 * col(0) + 0.99 * T1 * col(1)
    np.testing.assert_allclose(out["rgb"][j, i], want, atol=1e-12)
    np.testing.assert_allclose(out["T"][j, i], T2, rtol=1e-14)
    assert out["n_eval"][j, i] == 3 and out["n_alpha"][j, i] == 3


def test_alpha_threshold(orc):
    """Opacity just above / below 1/255 at the pixel: kept / skipped."""
    W, H, f = 16, 16, 20.0
    vm, it = identity_camera(W, H, f)
    for o, kept in [(1 / 255 * 1.02, True), (1 / 255 * 0.98, False)]:
        sc = scene_from([[0, 0, 2.0]], [math.log(1.0)] * 3, [1, 0, 0, 0], logit(o),
                        colours=(1, 1, 1))
        rec = orc.project(sc, vm, it, W, H)
        out = orc.render(sc, vm, it, W, H)
        a = rec["o"][0] * math.exp(-0.5 * rec["A"][0] * 0.5)  # pixel (8, 8): d = (0.5, 0.5)
        assert (a >= 1 / 255) == kept
        np.testing.assert_allclose(out["rgb"][8, 8, 0], rec["red"][0] * a if kept else 0.0,
                                   atol=1e-15)


def test_sum_of_weights_plus_T_is_one(orc):
    """Telescoping identity: with every colour c, red / c = sum_i w_i and
    red / c + T = 1 per pixel."""
    rng = np.random.default_rng(3)
    n = 400
    means = np.c_[rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(1, 4, n)]
    q = rng.normal(size=(n, 4))
    sc = scene_from(means, rng.normal(-2.5, 0.5, (n, 3)), q, rng.normal(0, 1.5, n),
                    colours=(1, 1, 1))
    vm, it = identity_camera(48, 40, 40.0)
    out = orc.render(sc, vm, it, 48, 40)
    c = 0.5 + Y00 * f32(dc_for_colour(1.0))  # the colour the float32 DC encodes
    s = out["rgb"][..., 0] / c + out["T"]
    assert np.abs(s - 1).max() < 1e-12
    assert (out["T"] < 1).sum() > 100  # something was drawn
    assert (out["T"] >= 1e-4 * 0.0099).all()


def test_bruteforce_equals_tiled(orc):
    rng = np.random.default_rng(4)
    for trial in range(4):
        n = 64
        means = np.c_[rng.uniform(-1.5, 1.5, n), rng.uniform(-1.5, 1.5, n), rng.uniform(0.5, 3, n)]
        sc = scene_from(means, rng.normal(-2, 0.6, (n, 3)), rng.normal(size=(n, 4)),
                        rng.normal(0, 2, n), colours=rng.uniform(0, 1, (n, 3)))
        vm, it = identity_camera(32, 32, 24.0)
        a = orc.render(sc, vm, it, 32, 32, mode="tiled")
        b = orc.render(sc, vm, it, 32, 32, mode="brute")
        for k in ("rgb", "depth", "T", "n_eval"):
            np.testing.assert_array_equal(a[k], b[k])


def test_rigid_motion_invariance(orc):
    """Moving the scene and the camera by the same rigid motion leaves a
    degree-0 render unchanged (pins the camera transform and quaternions)."""
    rng = np.random.default_rng(6)
    n = 300
    means = np.c_[rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(1.5, 4, n)]
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    ls = rng.normal(-2.5, 0.4, (n, 3))
    lo = rng.normal(0, 1, n)
    cols = rng.uniform(0, 1, (n, 3))
    W, H = 40, 32
    vm, it = identity_camera(W, H, 36.0)
    base = orc.render(scene_from(means, ls, q, lo, colours=cols), vm, it, W, H)
    Rm = Rotation.from_euler("xyz", [0.4, -0.9, 1.3])
    tvec = np.array([0.5, -2.0, 0.7])
    means2 = Rm.apply(means) + tvec
    rq = (Rm * Rotation.from_quat(q[:, [1, 2, 3, 0]])).as_quat()  # (x,y,z,w)
    q2 = rq[:, [3, 0, 1, 2]]
    M = np.eye(4)
    M[:3, :3] = Rm.as_matrix()
    M[:3, 3] = tvec
    vm2 = vm.astype(np.float64) @ np.linalg.inv(M)
    moved = orc.render(scene_from(means2, ls, q2, lo, colours=cols), vm2, it, W, H)
    # inputs are rounded to float32 in both scenes, so allow that much
    np.testing.assert_allclose(moved["rgb"], base["rgb"], atol=2e-4)
    np.testing.assert_allclose(moved["T"], base["T"], atol=2e-4)


def test_sh_view_direction(orc):
    """Degree-1 colour follows the camera->mean direction in world space."""
    W, H, f = 32, 32, 30.0
    sh = np.zeros((4, 3, 1))
    k = 0.8
    sh[2, :, 0] = k  # coefficient of Y_10 = C1 * dir_z
    mean = np.array([[0.0, 0.0, 2.0]])
    sc = scene_from(mean, [math.log(0.1)] * 3, [1, 0, 0, 0], 0.0, sh=sh, deg=1)
    # camera at (0, 0, 0) looking along +z: dir = (0, 0, 1)
    vm, it = identity_camera(W, H, f)
    rec = orc.project(sc, vm, it, W, H)
    C1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(rec["red"][0], 0.5 + f32(k) * C1, rtol=1e-12)
    # camera at (0, 0, 4) looking back along -z: dir = (0, 0, -1)
    V = np.diag([-1.0, 1.0, -1.0, 1.0])
    V[:3, 3] = -V[:3, :3] @ np.array([0.0, 0.0, 4.0])
    rec2 = orc.project(sc, V, it, W, H)
    np.testing.assert_allclose(rec2["red"][0], 0.5 - f32(k) * C1, rtol=1e-12)


# -------------------------------------------------------------- edge cases


def test_near_plane_and_behind(orc):
    W, H, f = 32, 32, 30.0
    vm, it = identity_camera(W, H, f)
    for z, visible in [(0.19, False), (0.21, True), (-1.0, False)]:
        sc = scene_from([[0, 0, z]], [math.log(0.02)] * 3, [1, 0, 0, 0], 2.0)
        out = orc.render(sc, vm, it, W, H)
        assert (out["T"].min() < 1) == visible, z


def test_camera_inside_gaussian_is_culled(orc):
    W, H, f = 32, 32, 30.0
    vm, it = identity_camera(W, H, f)
    sc = scene_from([[0, 0, 0.05]], [math.log(2.0)] * 3, [1, 0, 0, 0], 3.0)
    out = orc.render(sc, vm, it, W, H)
    assert (out["T"] == 1).all() and (out["rgb"] == 0).all()


def test_covering_all_tiles_and_partial_row(orc):
    W, H, f = 160, 120, 120.0  # TY = 8 with a partial last tile row
    vm, it = identity_camera(W, H, f)
    sc = scene_from([[0, 0, 1.0]], [math.log(0.5)] * 3, [1, 0, 0, 0], 0.0)
    rec = orc.project(sc, vm, it, W, H)
    assert list(rec["rect"][0]) == [0, 9, 0, 7]
    lists = orc.tile_lists(sc, vm, it, W, H)
    assert len(lists["g"]) == 80
    out = orc.render(sc, vm, it, W, H)
    assert out["rgb"].shape == (120, 160, 3)
    assert (out["T"] < 1).all()


def test_zero_survivors(orc):
    W, H, f = 32, 24, 30.0
    vm, it = identity_camera(W, H, f)
    sc = scene_from([[0, 0, -3.0], [10.0, 0, 1.0]], [math.log(0.05)] * 3, [1, 0, 0, 0], 0.0)
    assert orc.project(sc, vm, it, W, H)["n_valid"] == 0
    out = orc.render(sc, vm, it, W, H)
    assert (out["T"] == 1).all() and (out["rgb"] == 0).all() and (out["depth"] == 0).all()


def test_tile_lists_sorted_and_complete(orc):
    rng = np.random.default_rng(8)
    n = 200
    means = np.c_[rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(1, 3, n)]
    means[10, 2] = means[11, 2]  # an exact depth tie
    sc = scene_from(means, rng.normal(-2.5, 0.5, (n, 3)), rng.normal(size=(n, 4)), 0.0)
    W, H = 64, 48
    vm, it = identity_camera(W, H, 40.0)
    L = orc.tile_lists(sc, vm, it, W, H)
    rec = orc.project(sc, vm, it, W, H)
    TX = 4
    for t in range(12):
        g = L["g"][L["off"][t]:L["off"][t + 1]]
        want = [k for k in range(n) if rec["valid"][k] and
                rec["rect"][k][0] <= t % TX <= rec["rect"][k][1] and
                rec["rect"][k][2] <= t // TX <= rec["rect"][k][3]]
        assert sorted(g.tolist()) == want
        keys = [(rec["z"][k], k) for k in g]
        assert keys == sorted(keys)


def test_bands_report_flipped_alternative(orc):
    """A pixel whose alpha sits within the band of 1/255 gets an alternative
    result with the flipped decision, and the primary is among the leaves."""
    W, H, f = 16, 16, 20.0
    vm, it = identity_camera(W, H, f)
    o = 1 / 255 * 1.0001
    sc = scene_from([[0, 0, 2.0]], [math.log(1.0)] * 3, [1, 0, 0, 0], logit(o), colours=(1, 1, 1))
    bands = O.Bands(ln_alpha=5e-3, max_flips=2, max_leaves=8)
    out = orc.render(sc, vm, it, W, H, bands=bands)
    assert out["flags"][8, 8] & 1
    leaves = out["leaf_val"][out["leaf_pix"] == 8 * W + 8]
    reds = sorted(leaves[:, 0].tolist())
    assert len(reds) == 2 and reds[0] == 0.0 and reds[1] > 0
    assert out["rgb"][8, 8, 0] in reds
