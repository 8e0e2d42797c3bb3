"""Python binding of the C ABI in ``include/gs.h`` (argument marshalling only).

Functions keep the C names (``gs_context_create``, ``gs_scene_create``,
``gs_render_batch`` ...). ``Renderer`` is a thin convenience wrapper that takes
torch tensors and passes their device pointers and the current CUDA stream;
every step of the render runs in ``libgs_b300.so``. Importing this module
loads the library and raises if it is missing or was built for another ABI.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgs_b300.so")
ABI_VERSION = 6

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CUDA, GS_ERR_OOM, GS_ERR_CAPACITY, GS_ERR_TIMEOUT, \
    GS_ERR_NOT_FOUND = range(7)
GS_F32, GS_F16, GS_BF16 = 0, 1, 2
GS_MEM_HOST, GS_MEM_DEVICE = 0, 1


class gs_config(ctypes.Structure):
    _fields_ = [("near_plane", ctypes.c_float), ("dilation", ctypes.c_float),
                ("guard_band", ctypes.c_float), ("sigma_cull", ctypes.c_float),
                ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("T_min", ctypes.c_float), ("background", ctypes.c_float * 3),
                ("max_chunk_cameras", ctypes.c_int32), ("camera_group", ctypes.c_int32),
                ("count_pairs", ctypes.c_int32), ("time_stages", ctypes.c_int32),
                ("pixels_per_thread", ctypes.c_int32), ("tiles_per_block", ctypes.c_int32),
                ("workspace_survivors", ctypes.c_int64), ("sync_errors", ctypes.c_int32),
                ("comp_batch", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("depth_prefix", ctypes.c_int32)]


class gs_scene_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("geometry_dtype", ctypes.c_int32), ("appearance_dtype", ctypes.c_int32),
                ("memory", ctypes.c_int32), ("mean", ctypes.c_void_p),
                ("log_scale", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("logit_opacity", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class gs_stats(ctypes.Structure):
    _fields_ = [("n_cameras", ctypes.c_int64), ("survivors", ctypes.c_int64),
                ("intersections", ctypes.c_int64), ("pairs_evaluated", ctypes.c_int64),
                ("pairs_alpha", ctypes.c_int64), ("n_chunks", ctypes.c_int32),
                ("ms_project", ctypes.c_float), ("ms_sort", ctypes.c_float),
                ("ms_bin", ctypes.c_float), ("ms_composite", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("reserved0", ctypes.c_int32),
                ("warp_iters", ctypes.c_int64), ("warp_iters_box", ctypes.c_int64),
                ("warp_iters_blend", ctypes.c_int64), ("sort_windows_listed", ctypes.c_int64),
                ("sort_equal_runs", ctypes.c_int64), ("sort_long_runs", ctypes.c_int64),
                ("depth_second_phase_cameras", ctypes.c_int64),
                ("depth_resumed_tiles", ctypes.c_int64)]


# name -> (restype, argtypes); the same set as include/gs.h declares
_vp, _i32, _i64, _f32p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
SIGNATURES = {
    "gs_abi_version": (ctypes.c_int32, []),
    "gs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gs_config_default": (ctypes.c_int, [ctypes.POINTER(gs_config)]),
    "gs_context_create": (ctypes.c_int, [ctypes.POINTER(gs_config), _i32, ctypes.POINTER(_vp)]),
    "gs_context_set_config": (ctypes.c_int, [_vp, _vp]),
    "gs_context_destroy": (None, [_vp]),
    "gs_last_error": (ctypes.c_char_p, [_vp]),
    "gs_scene_create": (ctypes.c_int, [_vp, ctypes.POINTER(gs_scene_desc),
                                       ctypes.POINTER(ctypes.c_int32)]),
    "gs_scene_destroy": (ctypes.c_int, [_vp, _i32]),
    "gs_render_batch": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _i32, _i32, _vp, _vp, _vp,
                                       _vp]),
    "gs_render_batch_host": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _i32, _i32, _vp, _vp,
                                            _vp, _vp]),
    "gs_render_batch_v": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                         _vp]),
    "gs_render_motion_blur": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, ctypes.c_float,
                                             _i32, _i32, _i32, _vp, _vp, _vp, _vp]),
    "gs_graph_create": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                       ctypes.POINTER(_vp)]),
    "gs_graph_launch": (ctypes.c_int, [_vp, _vp]),
    "gs_graph_check": (ctypes.c_int, [_vp, _vp]),
    "gs_graph_destroy": (None, [_vp]),
    "gs_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(gs_stats)]),
    "gs_sync": (ctypes.c_int, [_vp, _vp]),
    "gs_render_timeout_probe": (ctypes.c_int, [_vp, _i32, _vp, _vp, _i32, _i32, _vp, _vp, _vp]),
    "gs_set_resume_capacity": (ctypes.c_int, [_vp, _i32]),
    "gs_debug_project": (ctypes.c_int, [_vp, _i32, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _i64,
                                        ctypes.POINTER(_i64), _vp]),
    "gs_debug_tile_lists": (ctypes.c_int, [_vp, _i32, _vp, _vp, _i32, _i32, _vp, _vp, _i64,
                                           ctypes.POINTER(_i64), _vp]),
    "gs_sort_segments": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _vp, _i32, _vp]),
    "gs_sort_segments_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _i32, _vp]),
    "gs_upsampler_param_count": (_i64, []),
    "gs_upsampler_create": (ctypes.c_int, [_i32, ctypes.POINTER(_vp)]),
    "gs_upsampler_destroy": (None, [_vp]),
    "gs_upsampler_last_error": (ctypes.c_char_p, [_vp]),
    "gs_upsampler_set_params": (ctypes.c_int, [_vp, _vp, _i64]),
    "gs_upsampler_get_params": (ctypes.c_int, [_vp, _vp, _i64]),
    "gs_upsampler_get_grads": (ctypes.c_int, [_vp, _vp, _i64]),
    "gs_upsample_forward": (ctypes.c_int, [_vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
    "gs_upsample_grad": (ctypes.c_int, [_vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp]),
    "gs_upsample_adam": (ctypes.c_int, [_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, _vp]),
    "gs_upsampler_set_backend": (ctypes.c_int, [_vp, _i32]),
    "gs_upsample_check": (ctypes.c_int, [_vp, _vp]),
    "gs_upsample_timeout_probe": (ctypes.c_int, [_vp, _vp]),
    "gs_render_batch_upsampled": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp, _vp, _i32, _i32, _vp,
                                                 _vp, _vp]),
    "gs_microbench": (ctypes.c_int, [_i32, _i32, _i32, _vp, _vp, _vp]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -m paper_2510_15352_b300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    v = lib.gs_abi_version()
    if v != ABI_VERSION:
        raise ImportError(f"libgs_b300.so ABI {v}, binding expects {ABI_VERSION}")
    return lib


lib = load()

# C-named entry points (same names, same arguments)
gs_abi_version = lib.gs_abi_version
gs_status_string = lib.gs_status_string
gs_config_default = lib.gs_config_default
gs_context_create = lib.gs_context_create
gs_context_destroy = lib.gs_context_destroy
gs_context_set_config = lib.gs_context_set_config
gs_last_error = lib.gs_last_error
gs_scene_create = lib.gs_scene_create
gs_scene_destroy = lib.gs_scene_destroy
gs_render_batch = lib.gs_render_batch
gs_render_batch_host = lib.gs_render_batch_host
gs_render_batch_v = lib.gs_render_batch_v
gs_render_motion_blur = lib.gs_render_motion_blur
gs_graph_create = lib.gs_graph_create
gs_graph_launch = lib.gs_graph_launch
gs_graph_check = lib.gs_graph_check
gs_graph_destroy = lib.gs_graph_destroy
gs_get_stats = lib.gs_get_stats
gs_sync = lib.gs_sync
gs_render_timeout_probe = lib.gs_render_timeout_probe
gs_set_resume_capacity = lib.gs_set_resume_capacity
gs_debug_project = lib.gs_debug_project
gs_debug_tile_lists = lib.gs_debug_tile_lists
gs_sort_segments = lib.gs_sort_segments
gs_sort_segments_noalloc = lib.gs_sort_segments_noalloc
gs_upsampler_param_count = lib.gs_upsampler_param_count
gs_upsampler_create = lib.gs_upsampler_create
gs_upsampler_destroy = lib.gs_upsampler_destroy
gs_upsampler_last_error = lib.gs_upsampler_last_error
gs_upsampler_set_params = lib.gs_upsampler_set_params
gs_upsampler_get_params = lib.gs_upsampler_get_params
gs_upsampler_get_grads = lib.gs_upsampler_get_grads
gs_upsample_forward = lib.gs_upsample_forward
gs_upsample_grad = lib.gs_upsample_grad
gs_upsample_adam = lib.gs_upsample_adam
gs_upsampler_set_backend = lib.gs_upsampler_set_backend
gs_upsample_check = lib.gs_upsample_check
gs_upsample_timeout_probe = lib.gs_upsample_timeout_probe
gs_render_batch_upsampled = lib.gs_render_batch_upsampled
gs_microbench = lib.gs_microbench
GS_UPSAMPLE_TCGEN05, GS_UPSAMPLE_MMA_SYNC = 0, 1


class GSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{gs_status_string(status).decode()}: {msg}")
        self.status = status


def default_config(**over) -> gs_config:
    c = gs_config()
    gs_config_default(ctypes.byref(c))
    for k, v in over.items():
        if k == "background":
            c.background[:] = list(v)
        else:
            setattr(c, k, v)
    return c


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


class Renderer:
    """A context plus its scenes. Tensors in, tensors out; the kernels do the work."""

    def __init__(self, device: int = 0, **config):
        self.cfg = default_config(**config)
        h = ctypes.c_void_p()
        st = gs_context_create(ctypes.byref(self.cfg), device, ctypes.byref(h))
        if st != GS_OK:
            raise GSError(st, "context creation")
        self.ctx = h
        self.device = device
        self.overrides = dict(config)

    def set_config(self, **config):
        """gs_context_set_config: new launch parameters (defaults for those not
        given), scenes and workspace kept."""
        cfg = default_config(**config)
        self._check(gs_context_set_config(self.ctx, ctypes.byref(cfg)))
        self.cfg = cfg
        self.overrides = dict(config)

    def close(self):
        if self.ctx:
            gs_context_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != GS_OK:
            raise GSError(st, gs_last_error(self.ctx).decode())

    # ------------------------------------------------------------- scenes
    def add_scene(self, scene: dict) -> int:
        """Upload a scene dict (numpy arrays or tensors, layout of gs.h).
        float16 arrays are taken as FP16, uint16 arrays as BF16 bit patterns."""
        arrs = [scene[k] for k in ("mean", "log_scale", "quat", "logit_opacity", "sh")]

        def kind(a):
            dt = str(a.dtype)
            if "float32" in dt:
                return GS_F32
            if "bfloat16" in dt or "uint16" in dt:
                return GS_BF16
            if "float16" in dt:
                return GS_F16
            raise TypeError(f"unsupported dtype {dt}")

        geo = {kind(a) for a in arrs[:3]}
        app = {kind(a) for a in arrs[3:]}
        if len(geo) != 1 or len(app) != 1:
            raise TypeError("mean/log_scale/quat and logit_opacity/sh must share a dtype")
        on_dev = hasattr(arrs[0], "is_cuda") and arrs[0].is_cuda
        if on_dev:
            arrs = [a.contiguous() for a in arrs]
            ptrs = [a.data_ptr() for a in arrs]
        else:
            arrs = [np.ascontiguousarray(a) for a in arrs]
            ptrs = [a.ctypes.data for a in arrs]
        d = gs_scene_desc(n=int(arrs[0].shape[-1]), sh_degree=int(scene["sh_degree"]),
                          geometry_dtype=geo.pop(), appearance_dtype=app.pop(),
                          memory=GS_MEM_DEVICE if on_dev else GS_MEM_HOST,
                          mean=ptrs[0], log_scale=ptrs[1], quat=ptrs[2],
                          logit_opacity=ptrs[3], sh=ptrs[4])
        sid = ctypes.c_int32()
        self._check(gs_scene_create(self.ctx, ctypes.byref(d), ctypes.byref(sid)))
        return sid.value

    def remove_scene(self, sid: int):
        self._check(gs_scene_destroy(self.ctx, sid))

    # ------------------------------------------------------------- render
    def render(self, scene_ids, viewmats, intrinsics, W: int, H: int, rgb=None, depth=None,
               final_T=None, want_T: bool = False, stream=None):
        """Render on the GPU. viewmats (n,4,4) / intrinsics (n,4) float32 CUDA
        tensors; outputs are allocated when not given. Returns (rgb, depth, T)."""
        import torch
        n = int(viewmats.shape[0])
        ids = np.ascontiguousarray(np.broadcast_to(np.asarray(scene_ids, dtype=np.int32), (n,)))
        dev = viewmats.device
        if rgb is None:
            rgb = torch.empty((n, H, W, 3), dtype=torch.float32, device=dev)
        if depth is None:
            depth = torch.empty((n, H, W), dtype=torch.float32, device=dev)
        if final_T is None and want_T:
            final_T = torch.empty((n, H, W), dtype=torch.float32, device=dev)
        vm = viewmats.contiguous()
        it = intrinsics.contiguous()
        self._check(gs_render_batch(self.ctx, n, ids.ctypes.data, vm.data_ptr(), it.data_ptr(),
                                    W, H, rgb.data_ptr(), depth.data_ptr(), _ptr(final_T),
                                    _stream(stream)))
        return rgb, depth, final_T

    def render_upsampled(self, upsampler: "Upsampler", scene_ids, viewmats, intrinsics, W: int,
                         H: int, rgb=None, depth=None, stream=None):
        """The upsampled path (gs_render_batch_upsampled): render at W/4 x H/4,
        upsample to W x H with `upsampler`. Returns (rgb, depth)."""
        import torch
        n = int(viewmats.shape[0])
        ids = np.ascontiguousarray(np.broadcast_to(np.asarray(scene_ids, dtype=np.int32), (n,)))
        dev = viewmats.device
        if rgb is None:
            rgb = torch.empty((n, H, W, 3), dtype=torch.float32, device=dev)
        if depth is None:
            depth = torch.empty((n, H, W), dtype=torch.float32, device=dev)
        vm = viewmats.contiguous()
        it = intrinsics.contiguous()
        self._check(gs_render_batch_upsampled(self.ctx, upsampler.u, n, ids.ctypes.data,
                                              vm.data_ptr(), it.data_ptr(), W, H, rgb.data_ptr(),
                                              depth.data_ptr(), _stream(stream)))
        return rgb, depth

    def render_v(self, scene_ids, viewmats, intrinsics, widths, heights, rgb=None, depth=None,
                 final_T=None, want_T: bool = False, stream=None):
        """Render cameras of mixed sizes into packed outputs (camera i's pixels
        start at offsets[i]). Returns (rgb [P, 3], depth [P], T or None, offsets)."""
        import torch
        n = int(viewmats.shape[0])
        ids = np.ascontiguousarray(np.broadcast_to(np.asarray(scene_ids, dtype=np.int32), (n,)))
        w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
        h = np.ascontiguousarray(np.asarray(heights, dtype=np.int32))
        sizes = w.astype(np.int64) * h
        off = np.ascontiguousarray(np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64))
        P = int(sizes.sum())
        dev = viewmats.device
        if rgb is None:
            rgb = torch.empty((P, 3), dtype=torch.float32, device=dev)
        if depth is None:
            depth = torch.empty((P,), dtype=torch.float32, device=dev)
        if final_T is None and want_T:
            final_T = torch.empty((P,), dtype=torch.float32, device=dev)
        vm = viewmats.contiguous()
        it = intrinsics.contiguous()
        self._check(gs_render_batch_v(self.ctx, n, ids.ctypes.data, vm.data_ptr(), it.data_ptr(),
                                      w.ctypes.data, h.ctypes.data, off.ctypes.data,
                                      rgb.data_ptr(), depth.data_ptr(), _ptr(final_T),
                                      _stream(stream)))
        return rgb, depth, final_T, off

    def graph(self, scene_ids, viewmats, intrinsics, widths, heights, rgb, depth, final_T=None):
        """Capture the render of these cameras into a CUDA graph (outputs packed as
        in render_v, which must be preallocated). Returns a Graph."""
        n = int(viewmats.shape[0])
        ids = np.ascontiguousarray(np.broadcast_to(np.asarray(scene_ids, dtype=np.int32), (n,)))
        w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
        h = np.ascontiguousarray(np.asarray(heights, dtype=np.int32))
        sizes = w.astype(np.int64) * h
        off = np.ascontiguousarray(np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64))
        g = ctypes.c_void_p()
        self._check(gs_graph_create(self.ctx, n, ids.ctypes.data, viewmats.data_ptr(),
                                    intrinsics.data_ptr(), w.ctypes.data, h.ctypes.data,
                                    off.ctypes.data, rgb.data_ptr(), depth.data_ptr(),
                                    _ptr(final_T), ctypes.byref(g)))
        return Graph(self, g, off)

    def render_motion_blur(self, scene_ids, viewmats, intrinsics, velocities, shutter: float,
                           samples: int, W: int, H: int, want_T: bool = False, stream=None):
        """Motion-blurred render (device tensors in and out). Returns (rgb, depth, T)."""
        import torch
        n = int(viewmats.shape[0])
        ids = np.ascontiguousarray(np.broadcast_to(np.asarray(scene_ids, dtype=np.int32), (n,)))
        dev = viewmats.device
        rgb = torch.empty((n, H, W, 3), dtype=torch.float32, device=dev)
        depth = torch.empty((n, H, W), dtype=torch.float32, device=dev)
        T = torch.empty((n, H, W), dtype=torch.float32, device=dev) if want_T else None
        vm, it, vel = viewmats.contiguous(), intrinsics.contiguous(), velocities.contiguous()
        self._check(gs_render_motion_blur(self.ctx, n, ids.ctypes.data, vm.data_ptr(),
                                          it.data_ptr(), vel.data_ptr(), float(shutter),
                                          int(samples), W, H, rgb.data_ptr(), depth.data_ptr(),
                                          _ptr(T), _stream(stream)))
        return rgb, depth, T

    def render_host(self, scene_ids, viewmats, intrinsics, W: int, H: int, rgb, depth,
                    final_T=None, stream=None):
        """Render with every array in host memory (pinned tensors copy fastest)."""
        n = int(viewmats.shape[0])
        ids = np.ascontiguousarray(np.broadcast_to(np.asarray(scene_ids, dtype=np.int32), (n,)))
        self._check(gs_render_batch_host(self.ctx, n, ids.ctypes.data, viewmats.data_ptr(),
                                         intrinsics.data_ptr(), W, H, rgb.data_ptr(),
                                         depth.data_ptr(), _ptr(final_T), _stream(stream)))
        return rgb, depth, final_T

    def timeout_probe(self, sid: int, viewmat, intr, W: int, H: int, stream=None) -> int:
        """gs_render_timeout_probe: the status it returns (GS_ERR_TIMEOUT expected)."""
        import torch
        rgb = torch.empty((1, H, W, 3), dtype=torch.float32, device=viewmat.device)
        depth = torch.empty((1, H, W), dtype=torch.float32, device=viewmat.device)
        return int(gs_render_timeout_probe(self.ctx, sid, viewmat.data_ptr(), intr.data_ptr(), W, H,
                                           rgb.data_ptr(), depth.data_ptr(), _stream(stream)))

    def set_resume_capacity(self, tiles: int) -> None:
        """gs_set_resume_capacity: cap the first phase's saved-state list (0: default)."""
        self._check(gs_set_resume_capacity(self.ctx, tiles))

    def sync(self, stream=None) -> None:
        """gs_sync: wait for the stream and the last render call; raise a
        pending device-detected error of an earlier call."""
        self._check(gs_sync(self.ctx, _stream(stream)))

    def stats(self) -> dict:
        s = gs_stats()
        self._check(gs_get_stats(self.ctx, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in gs_stats._fields_ if not k.startswith("reserved")}

    # ------------------------------------------------------------- inspection
    def debug_project(self, sid: int, viewmat, intr, W: int, H: int, cap: int):
        rec = np.zeros((cap, 12), dtype=np.float32)
        gidx = np.zeros(cap, dtype=np.int32)
        rect = np.zeros((cap, 4), dtype=np.int32)
        n = ctypes.c_int64()
        self._check(gs_debug_project(self.ctx, sid, viewmat.data_ptr(), intr.data_ptr(), W, H,
                                     rec.ctypes.data, gidx.ctypes.data, rect.ctypes.data, cap,
                                     ctypes.byref(n), _stream(None)))
        k = n.value
        return rec[:k], gidx[:k], rect[:k]

    def debug_tile_lists(self, sid: int, viewmat, intr, W: int, H: int, cap: int):
        ntiles = ((W + 15) // 16) * ((H + 15) // 16)
        off = np.zeros(ntiles + 1, dtype=np.int64)
        gidx = np.zeros(max(cap, 1), dtype=np.int32)
        n = ctypes.c_int64()
        self._check(gs_debug_tile_lists(self.ctx, sid, viewmat.data_ptr(), intr.data_ptr(), W,
                                        H, off.ctypes.data, gidx.ctypes.data, cap,
                                        ctypes.byref(n), _stream(None)))
        return off, gidx[:n.value]

    def sort_segments(self, keys, vals, seg_start, seg_count, stream=None):
        """In-place stable segmented sort of uint32 keys (int32 tensors hold the bits)."""
        self._check(gs_sort_segments(self.ctx, keys.data_ptr(), vals.data_ptr(), keys.numel(),
                                     seg_start.data_ptr(), seg_count.data_ptr(),
                                     int(seg_start.numel()), _stream(stream)))


class Graph:
    """A captured render: launch() replays it on a stream; check() waits and
    reports a workspace overflow of the last replay."""

    def __init__(self, renderer: Renderer, handle, offsets):
        self.r = renderer
        self.h = handle
        self.offsets = offsets

    def launch(self, stream=None):
        self.r._check(gs_graph_launch(self.h, _stream(stream)))

    def check(self, stream=None):
        self.r._check(gs_graph_check(self.h, _stream(stream)))

    def close(self):
        if self.h:
            gs_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Upsampler:
    """The learned 4x upsampler (gs_upsampler_*): parameters, inference, one
    training pass and Adam. Tensors are CUDA float32, NHWC, contiguous."""

    n_params = int(gs_upsampler_param_count())

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        st = gs_upsampler_create(device, ctypes.byref(h))
        if st != GS_OK:
            raise GSError(st, "upsampler creation")
        self.u = h
        self.device = device

    def close(self):
        if self.u:
            gs_upsampler_destroy(self.u)
            self.u = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != GS_OK:
            raise GSError(st, gs_upsampler_last_error(self.u).decode())

    def set_params(self, flat) -> None:
        a = np.ascontiguousarray(flat, dtype=np.float32).ravel()
        self._check(gs_upsampler_set_params(self.u, a.ctypes.data, a.size))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.n_params, np.float32)
        self._check(gs_upsampler_get_params(self.u, a.ctypes.data, a.size))
        return a

    def get_grads(self) -> np.ndarray:
        a = np.empty(self.n_params, np.float32)
        self._check(gs_upsampler_get_grads(self.u, a.ctypes.data, a.size))
        return a

    def forward(self, lr_rgb, lr_depth=None, out_rgb=None, out_depth=None, stream=None):
        import torch
        n, h, w, _ = lr_rgb.shape
        if out_rgb is None:
            out_rgb = torch.empty((n, 4 * h, 4 * w, 3), dtype=torch.float32, device=lr_rgb.device)
        if lr_depth is not None and out_depth is None:
            out_depth = torch.empty((n, 4 * h, 4 * w), dtype=torch.float32, device=lr_rgb.device)
        self._check(gs_upsample_forward(self.u, n, h, w, _ptr(lr_rgb), _ptr(lr_depth),
                                        _ptr(out_rgb), _ptr(out_depth), _stream(stream)))
        return out_rgb, out_depth

    def grad(self, lr_rgb, hr_target, loss=None, stream=None):
        import torch
        n, h, w, _ = lr_rgb.shape
        if loss is None:
            loss = torch.empty((1,), dtype=torch.float32, device=lr_rgb.device)
        self._check(gs_upsample_grad(self.u, n, h, w, _ptr(lr_rgb), _ptr(hr_target), _ptr(loss),
                                     _stream(stream)))
        return loss

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
             stream=None) -> None:
        self._check(gs_upsample_adam(self.u, lr, beta1, beta2, eps, _stream(stream)))

    def set_backend(self, backend: str) -> None:
        """"tcgen05" (default) or "mma_sync": the kernels of forward()."""
        code = {"tcgen05": GS_UPSAMPLE_TCGEN05, "mma_sync": GS_UPSAMPLE_MMA_SYNC}[backend]
        self._check(gs_upsampler_set_backend(self.u, code))

    def check(self, stream=None) -> None:
        """Synchronise and raise if a tensor-core kernel timed out."""
        self._check(gs_upsample_check(self.u, _stream(stream)))
