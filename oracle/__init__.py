"""FP64 CPU oracle for batched 3D Gaussian Splatting rendering.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. It shares no code with the CUDA path (``paper_2510_15352_b300``) and
imports nothing from it; both sides only share the seeded input generators of
``paper_2510_15352_b300.synth``, which hold none of the method's arithmetic.

The arithmetic lives in ``gs_oracle.c`` (plain C, double precision, OpenMP
over tiles); this module builds it with gcc and wraps it with ctypes.
What it computes is the renderer the paper drops into its simulator
(Sec. 3.2; depth as a by-product of compositing, Fig. 4): the cited 3DGS
rasteriser with EWA projection, 0.3 px dilation, 3-sigma tile culling,
16x16 tiles, (depth, index) order and front-to-back alpha compositing.

Every function is pinned by ``tests/test_oracle_pins.py`` (closed forms,
invariants, brute force, textbook SH) and ``tests/test_oracle_mutants.py``
(planted mistakes must fail a pin); the motion-blur poses and blend by
``tests/test_oracle_blur.py`` (camera centres recovered from the poses,
closed-form sub-frame images of one Gaussian, blend weights; planted
mistakes in copies of both functions must fail one of those pins).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "gs_oracle.c")
LIB = os.path.join(_HERE, "libgs_oracle.so")

R_FIELDS = ["u", "v", "z", "o", "A", "B", "C", "r", "a", "b", "c", "red", "green", "blue",
            "px", "py", "lmax", "det"]
R_COUNT = 20
ST_VALID, ST_AMBIG, ST_PROJ = 1, 2, 4


@dataclass
class Params:
    """Rendering constants (the rasteriser's fixed constants)."""
    near: float = 0.2
    dilation: float = 0.3
    guard: float = 1.3
    sigma: float = 3.0
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)
    tile: int = 16

    def array(self) -> np.ndarray:
        return np.array([self.near, self.dilation, self.guard, self.sigma, self.alpha_min,
                         self.alpha_max, self.T_min, self.bg[0], self.bg[1], self.bg[2],
                         float(self.tile)], dtype=np.float64)


@dataclass
class Bands:
    """Near-threshold bands; all zero gives the plain definition.

    px_abs/px_rel: tile-rect and off-image bounds (pixels; rel x (|u|+|v|+r));
    z_abs/z_rel: near plane and depth order (metres; rel x z);
    ln_alpha: |ln(o e^power) - ln(alpha_min)|; T_rel: |T' - T_min| / T_min.
    """
    px_abs: float = 0.0
    px_rel: float = 0.0
    z_abs: float = 0.0
    z_rel: float = 0.0
    ln_alpha: float = 0.0
    T_rel: float = 0.0
    max_flips: int = 0
    max_leaves: int = 1

    def array(self) -> np.ndarray:
        return np.array([self.px_abs, self.px_rel, self.z_abs, self.z_rel, self.ln_alpha,
                         self.T_rel, float(self.max_flips), float(self.max_leaves)],
                        dtype=np.float64)


def build(src: str = SRC, out: str = LIB, extra_flags=(), force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no FMA contraction)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           *extra_flags, src, "-o", out + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Oracle:
    """ctypes front end of ``gs_oracle.c``. ``lib_path`` selects another build
    (the mutant tests load planted-mistake builds through it)."""

    def __init__(self, lib_path: str | None = None):
        if lib_path is None:
            lib_path = build()
        self.lib = ctypes.CDLL(lib_path)
        L = self.lib
        L.or_abi_version.restype = ctypes.c_int
        L.or_sh_basis.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, _d]
        L.or_quat_to_rot.argtypes = [_d, _d]
        L.or_cov3d.argtypes = [_d, _d, _d]
        scene = [ctypes.c_int64, ctypes.c_int, _d, _d, _d, _d, _d, _d, _d, ctypes.c_int,
                 ctypes.c_int, _d, _d]
        L.or_project.argtypes = scene + [_d, _i32, _i32]
        L.or_project.restype = ctypes.c_int64
        L.or_tile_lists.argtypes = scene + [_i64, _i64, _i32, _d]
        L.or_tile_lists.restype = ctypes.c_int64
        L.or_render.argtypes = scene + [ctypes.c_int, _d, _d, _d, _i32, _i32, _i32,
                                        ctypes.c_int64, _i32, _d]
        L.or_render.restype = ctypes.c_int64

    # ---------------------------------------------------------------- pieces
    def sh_basis(self, deg: int, dirs) -> np.ndarray:
        dirs = _f64(dirs).reshape(-1, 3)
        K = (deg + 1) ** 2
        out = np.zeros((dirs.shape[0], 16), dtype=np.float64)
        for i, (x, y, z) in enumerate(dirs):
            self.lib.or_sh_basis(deg, x, y, z, _p(out[i], _d))
        return out[:, :K]

    def quat_to_rot(self, q) -> np.ndarray:
        q = _f64(q)
        R = np.zeros(9)
        self.lib.or_quat_to_rot(_p(q, _d), _p(R, _d))
        return R.reshape(3, 3)

    def cov3d(self, log_scale, q) -> np.ndarray:
        ls, q = _f64(log_scale), _f64(q)
        S = np.zeros(9)
        self.lib.or_cov3d(_p(ls, _d), _p(q, _d), _p(S, _d))
        return S.reshape(3, 3)

    # ----------------------------------------------------------------- scene
    @staticmethod
    def _scene_args(scene):
        mean = _f64(scene["mean"])
        n = mean.shape[1]
        deg = int(scene["sh_degree"])
        ls = _f64(scene["log_scale"])
        q = _f64(scene["quat"])
        lo = _f64(scene["logit_opacity"])
        sh = _f64(scene["sh"])
        assert mean.shape == (3, n) and ls.shape == (3, n) and q.shape == (4, n)
        assert lo.shape == (n,) and sh.shape == ((deg + 1) ** 2, 3, n)
        return n, deg, (mean, ls, q, lo, sh)

    def _common(self, scene, viewmat, intr, W, H, params, bands):
        n, deg, keep = self._scene_args(scene)
        vm = _f64(viewmat).reshape(16)
        it = _f64(intr).reshape(4)
        pa = (params or Params()).array()
        ba = (bands or Bands()).array()
        keep = keep + (vm, it, pa, ba)
        args = [n, deg] + [_p(a, _d) for a in keep[:5]] + [_p(vm, _d), _p(it, _d), int(W),
                                                           int(H), _p(pa, _d), _p(ba, _d)]
        return n, args, keep

    def project(self, scene, viewmat, intr, W, H, params=None, bands=None) -> dict:
        """Per-Gaussian projected records of one camera (double precision)."""
        n, args, keep = self._common(scene, viewmat, intr, W, H, params, bands)
        rec = np.zeros((max(n, 1), R_COUNT))
        rects = np.zeros((max(n, 1), 12), dtype=np.int32)
        status = np.zeros(max(n, 1), dtype=np.int32)
        nvalid = self.lib.or_project(*args, _p(rec, _d), _p(rects, _i32), _p(status, _i32))
        out = {k: rec[:n, i] for i, k in enumerate(R_FIELDS)}
        out["rect"] = rects[:n, 0:4]
        out["rect_ext"] = rects[:n, 4:8]
        out["rect_inner"] = rects[:n, 8:12]
        out["status"] = status[:n]
        out["valid"] = (status[:n] & ST_VALID) != 0
        out["n_valid"] = int(nvalid)
        return out

    def tile_lists(self, scene, viewmat, intr, W, H, params=None, bands=None) -> dict:
        """Per-tile (extended) lists in (depth, index) order with flags
        (bit0 member, bit1 ambiguous membership, bit2 depth-close to next)."""
        n, args, keep = self._common(scene, viewmat, intr, W, H, params, bands)
        tile = (params or Params()).tile
        ntiles = ((W + tile - 1) // tile) * ((H + tile - 1) // tile)
        total = self.lib.or_tile_lists(*args, None, None, None, None)
        if total < 0:
            raise MemoryError("oracle tile lists")
        off = np.zeros(ntiles + 1, dtype=np.int64)
        g = np.zeros(max(total, 1), dtype=np.int64)
        fl = np.zeros(max(total, 1), dtype=np.int32)
        z = np.zeros(max(total, 1))
        t2 = self.lib.or_tile_lists(*args, _p(off, _i64), _p(g, _i64), _p(fl, _i32), _p(z, _d))
        assert t2 == total
        return {"off": off, "g": g[:total], "flags": fl[:total], "z": z[:total]}

    def render(self, scene, viewmat, intr, W, H, params=None, bands=None,
               mode: str = "tiled") -> dict:
        """Render one camera. Returns rgb (H,W,3), depth, T, flags, n_eval,
        n_alpha and the alternative results of near-threshold pixels."""
        n, args, keep = self._common(scene, viewmat, intr, W, H, params, bands)
        m = {"tiled": 0, "brute": 1}[mode]
        rgb = np.zeros((H, W, 3))
        depth = np.zeros((H, W))
        T = np.zeros((H, W))
        flags = np.zeros((H, W), dtype=np.int32)
        n_eval = np.zeros((H, W), dtype=np.int32)
        n_alpha = np.zeros((H, W), dtype=np.int32)
        cap = max(1024, H * W // 4)
        while True:
            lp = np.zeros(cap, dtype=np.int32)
            lv = np.zeros((cap, 5))
            tot = self.lib.or_render(*args, m, _p(rgb, _d), _p(depth, _d), _p(T, _d),
                                     _p(flags, _i32), _p(n_eval, _i32), _p(n_alpha, _i32),
                                     cap, _p(lp, _i32), _p(lv, _d))
            if tot < 0:
                raise MemoryError("oracle render")
            if tot <= cap:
                break
            cap = int(tot)
        return {"rgb": rgb, "depth": depth, "T": T, "flags": flags, "n_eval": n_eval,
                "n_alpha": n_alpha, "leaf_pix": lp[:tot], "leaf_val": lv[:tot]}


def blur_poses(viewmat, velocity, shutter: float, samples: int) -> list:
    """Motion-blur sub-frame poses (Sec. 3.3, Fig. 9: frames offset along the
    camera's velocity, then blended): frame j moves the camera centre by
    velocity * shutter * (j/(samples-1) - 1/2), orientation kept, so the
    world->camera translation becomes t - R d. Double precision."""
    V = _f64(viewmat).reshape(4, 4)
    R, t = V[:3, :3], V[:3, 3]
    v = _f64(velocity).reshape(3)
    out = []
    for j in range(samples):
        frac = j / (samples - 1) - 0.5 if samples > 1 else 0.0
        W = V.copy()
        W[:3, 3] = t - R @ (v * shutter * frac)
        out.append(W)
    return out


def render_motion_blur(orc: "Oracle", scene, viewmat, intr, velocity, shutter: float,
                       samples: int, W: int, H: int, params=None, bands=None) -> dict:
    """Equal-weight blend of the sub-frame renders (rgb, depth and T). For each
    pixel, `allow` bounds how far a float32 renderer may drift from the blend
    through near-threshold decisions: the mean over sub-frames of the largest
    gap between that sub-frame's alternative results and its primary one."""
    acc = None
    for V in blur_poses(viewmat, velocity, shutter, samples):
        r = orc.render(scene, V, intr, W, H, params, bands)
        gap = np.zeros((H, W))
        if len(r["leaf_pix"]):
            prim = np.concatenate([r["rgb"].reshape(-1, 3), r["depth"].reshape(-1, 1),
                                   r["T"].reshape(-1, 1)], axis=1)
            d = np.abs(r["leaf_val"] - prim[r["leaf_pix"]]).max(axis=1)
            np.maximum.at(gap.reshape(-1), r["leaf_pix"], d)
        part = {"rgb": r["rgb"], "depth": r["depth"], "T": r["T"], "allow": gap}
        if acc is None:
            acc = {k: v / samples for k, v in part.items()}
        else:
            for k in acc:
                acc[k] = acc[k] + part[k] / samples
    return acc


_default = None


def get() -> Oracle:
    """Shared instance of the default build."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default
