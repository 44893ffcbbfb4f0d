"""Python binding of libhigs.so (argument marshalling only).

Every step of the render path runs in the library's CUDA kernels; this module
only converts torch tensors / numpy arrays into the C ABI's pointers and
structs (include/higs.h).  It fails loudly when the library cannot be loaded:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhigs.so")

HG_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error", -4: "capacity",
          -5: "device timeout", -6: "busy", -7: "not found", -8: "cancelled", -9: "unsupported"}
PATH_HIGS, PATH_PLAIN = 0, 1
BIN_RECT, BIN_ELLIPSE = 0, 1
FLAG_ASYNC, FLAG_TIMING, FLAG_KEEP_SPLATS, FLAG_INDEPENDENT, FLAG_PROFILE, FLAG_FP16 = 1, 2, 4, 8, 16, 32
(BUF_SEG_OFF, BUF_PAIR_KEYS, BUF_PAIR_IDS, BUF_BATCHES, BUF_SPLATS, BUF_VIEW_SEG_BASE, BUF_PLAIN_KEYS, BUF_PLAIN_IDS,
 BUF_TILE_RANGES, BUF_GRAD2D, BUF_RECORDS, BUF_VISIBILITY) = range(12)

EXPORTS = ["hg_status_str", "hg_last_error", "hg_version", "hg_ctx_create", "hg_ctx_destroy",
           "hg_create_scene", "hg_destroy_scene", "hg_scene_size", "hg_render", "hg_render_splats",
           "hg_state_free", "hg_state_sync", "hg_render_stats", "hg_state_read", "hg_graph_create",
           "hg_graph_launch", "hg_graph_set_cameras", "hg_graph_sync", "hg_graph_kernels", "hg_graph_destroy",
           "hg_kernel_launches", "hg_segmented_sort_noalloc", "hg_render_backward", "hg_autotune",
           "hg_serve_create", "hg_serve_add_scene", "hg_serve_submit", "hg_serve_poll", "hg_serve_wait",
           "hg_serve_cancel", "hg_serve_stats", "hg_serve_reset_stats", "hg_serve_destroy", "hg_l2_loss",
           "hg_adam_step", "hg_scene_sh_codec", "hg_spatial_order", "hg_scene_order", "hg_ctx_set_wait_limits"]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class AllocatorC(C.Structure):
    """hg_allocator: device memory callbacks of a context."""
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class AdamOpts(C.Structure):
    _fields_ = [("lr", C.c_float * 5), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int32)]


class HgError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SceneDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("borrow", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("sh_storage", C.c_int32),
                ("order", C.c_int32)]


SH_F32, SH_F16, SH_BF16, SH_CODEC32 = 0, 1, 2, 3
ORDER_INPUT, ORDER_SPATIAL = 0, 1


class CameraC(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class RenderOpts(C.Structure):
    _fields_ = [("path", C.c_int32), ("macro_w", C.c_int32), ("macro_h", C.c_int32),
                ("batch_cap", C.c_int32), ("bin_test", C.c_int32), ("bg", C.c_float * 3),
                ("save_for_backward", C.c_int32), ("flags", C.c_int32)]


class ServeConfig(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("max_views_per_launch", C.c_int32), ("mem_budget_bytes", C.c_int64),
                ("batch_window_us", C.c_int32), ("presize_width", C.c_int32), ("presize_height", C.c_int32),
                ("pad", C.c_int32), ("opts", RenderOpts)]


class ServeStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("submitted", "completed", "rejected", "cancelled", "failed", "launches",
                                          "queued", "inflight_launches", "max_inflight_seen", "held_bytes")] + \
               [(k, C.c_double) for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "req_per_s",
                                           "mean_views_per_launch")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneResult(C.Structure):
    _fields_ = [("macro_w", C.c_int32), ("macro_h", C.c_int32), ("batch_cap", C.c_int32), ("ms", C.c_float)]


class FrameStats(C.Structure):
    _fields_ = [("n_views", C.c_int64), ("n_gaussians", C.c_int64), ("n_visible", C.c_int64),
                ("n_pairs", C.c_int64), ("n_segments", C.c_int64), ("n_batches", C.c_int64),
                ("max_segment", C.c_int64), ("seg_by_tier", C.c_int64 * 6), ("n_sort_tiles", C.c_int64),
                ("n_replays", C.c_int64), ("raster_evals", C.c_int64), ("status", C.c_int32),
                ("sort_resorts", C.c_int32), ("ms_project", C.c_float), ("ms_partition", C.c_float),
                ("ms_sort", C.c_float), ("ms_raster", C.c_float), ("ms_merge", C.c_float),
                ("ms_total", C.c_float), ("raster_cycles", C.c_int64 * 6), ("pixel_support_evals", C.c_int64),
                ("pixel_contrib_evals", C.c_int64), ("pixel_live_evals", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("seg_by_tier", "raster_cycles")}
        d["seg_by_tier"] = list(self.seg_by_tier)
        d["raster_cycles"] = list(self.raster_cycles)
        return d


SPLAT_DTYPE = np.dtype([("mean2d", "<f4", 2), ("conic", "<f4", 3), ("opacity", "<f4"), ("rgb", "<f4", 3),
                        ("depth_key", "<u4"), ("radius", "<i4"), ("depth", "<f4")])
assert SPLAT_DTYPE.itemsize == 48

_lib = None


def load(path: str = LIB_PATH):
    """Load libhigs.so (raises if it is missing or lacks an exported symbol)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhigs.so not built ({path}); run paper_2606_00352_gb300/build.py")
    lib = C.CDLL(path)
    for name in EXPORTS:
        if not hasattr(lib, name):
            raise RuntimeError(f"libhigs.so does not export {name}")
    lib.hg_status_str.restype = C.c_char_p
    lib.hg_last_error.restype = C.c_char_p
    lib.hg_version.restype = C.c_char_p
    lib.hg_scene_size.restype = C.c_int64
    for name in ("hg_ctx_create", "hg_create_scene", "hg_render", "hg_render_splats",
                 "hg_state_sync", "hg_render_stats", "hg_state_read", "hg_graph_create", "hg_graph_launch",
                 "hg_graph_set_cameras", "hg_graph_sync"):
        getattr(lib, name).restype = C.c_int
    lib.hg_graph_create.argtypes = [C.c_void_p, C.POINTER(CameraC), C.c_int, C.POINTER(RenderOpts), C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]
    lib.hg_graph_launch.argtypes = [C.c_void_p, C.c_void_p]
    lib.hg_graph_set_cameras.argtypes = [C.c_void_p, C.POINTER(CameraC), C.c_int]
    lib.hg_graph_sync.argtypes = [C.c_void_p]
    lib.hg_graph_kernels.argtypes = [C.c_void_p]
    lib.hg_graph_kernels.restype = C.c_int64
    lib.hg_graph_destroy.argtypes = [C.c_void_p]
    lib.hg_kernel_launches.restype = C.c_int64
    for name in ("hg_serve_create", "hg_serve_add_scene", "hg_serve_submit", "hg_serve_poll", "hg_serve_wait",
                 "hg_serve_cancel", "hg_serve_stats", "hg_serve_reset_stats"):
        getattr(lib, name).restype = C.c_int
    lib.hg_serve_create.argtypes = [C.c_void_p, C.POINTER(ServeConfig), C.POINTER(C.c_void_p)]
    lib.hg_serve_add_scene.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
    lib.hg_serve_submit.argtypes = [C.c_void_p, C.c_int, C.POINTER(CameraC), C.c_void_p, C.c_int,
                                    C.POINTER(C.c_uint64)]
    lib.hg_serve_poll.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(C.c_int)]
    lib.hg_serve_wait.argtypes = [C.c_void_p, C.c_uint64, C.c_int]
    lib.hg_serve_cancel.argtypes = [C.c_void_p, C.c_uint64]
    lib.hg_serve_stats.argtypes = [C.c_void_p, C.POINTER(ServeStats)]
    lib.hg_serve_reset_stats.argtypes = [C.c_void_p]
    lib.hg_serve_destroy.argtypes = [C.c_void_p]
    lib.hg_autotune.restype = C.c_int
    lib.hg_autotune.argtypes = [C.c_void_p, C.POINTER(CameraC), C.c_int, C.POINTER(RenderOpts), C.c_int, C.c_char_p,
                                C.POINTER(RenderOpts), C.POINTER(TuneResult), C.c_int, C.POINTER(C.c_int), C.c_void_p]
    lib.hg_render_backward.restype = C.c_int
    lib.hg_render_backward.argtypes = [C.c_void_p] + [C.c_void_p] * 7
    lib.hg_scene_sh_codec.restype = C.c_int
    lib.hg_scene_sh_codec.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.hg_spatial_order.restype = C.c_int
    lib.hg_spatial_order.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    lib.hg_scene_order.restype = C.c_int
    lib.hg_scene_order.argtypes = [C.c_void_p, C.c_void_p]
    lib.hg_l2_loss.restype = C.c_int
    lib.hg_l2_loss.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.hg_adam_step.restype = C.c_int
    lib.hg_adam_step.argtypes = [C.c_void_p, C.c_void_p * 5, C.c_void_p * 5, C.c_void_p * 5, C.POINTER(AdamOpts),
                                 C.c_void_p]
    lib.hg_segmented_sort_noalloc.restype = C.c_int
    lib.hg_segmented_sort_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_void_p]
    lib.hg_ctx_create.argtypes = [C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
    lib.hg_ctx_set_wait_limits.restype = C.c_int
    lib.hg_ctx_set_wait_limits.argtypes = [C.c_void_p, C.c_int64, C.c_int64]
    lib.hg_ctx_destroy.argtypes = [C.c_void_p]
    lib.hg_create_scene.argtypes = [C.c_void_p, C.POINTER(SceneDesc), C.POINTER(C.c_void_p)]
    lib.hg_destroy_scene.argtypes = [C.c_void_p]
    lib.hg_scene_size.argtypes = [C.c_void_p]
    lib.hg_render.argtypes = [C.c_void_p, C.POINTER(CameraC), C.c_int, C.POINTER(RenderOpts), C.c_void_p,
                              C.c_void_p, C.POINTER(C.c_void_p), C.c_void_p]
    lib.hg_render_splats.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(CameraC), C.c_int,
                                     C.POINTER(RenderOpts), C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p),
                                     C.c_void_p]
    lib.hg_state_free.argtypes = [C.c_void_p]
    lib.hg_state_sync.argtypes = [C.c_void_p]
    lib.hg_render_stats.argtypes = [C.c_void_p, C.POINTER(FrameStats)]
    lib.hg_state_read.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]
    _lib = lib
    return lib


def check(status: int):
    if status != HG_OK:
        raise HgError(status, load().hg_last_error().decode())


def _stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def camera_struct(cam) -> CameraC:
    c = CameraC()
    vm = np.asarray(cam.viewmat, np.float32).reshape(16)
    for i in range(16):
        c.viewmat[i] = float(vm[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def cameras_array(cams):
    arr = (CameraC * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


@dataclass
class Options:
    path: int = PATH_HIGS
    macro_w: int = 8
    macro_h: int = 4
    batch_cap: int = 1024
    bin_test: int = BIN_RECT
    bg: tuple = (0.0, 0.0, 0.0)
    save_for_backward: bool = False
    flags: int = 0

    def struct(self) -> RenderOpts:
        o = RenderOpts()
        o.path, o.macro_w, o.macro_h, o.batch_cap, o.bin_test = (self.path, self.macro_w, self.macro_h,
                                                                 self.batch_cap, self.bin_test)
        for i in range(3):
            o.bg[i] = float(self.bg[i])
        o.save_for_backward = int(self.save_for_backward)
        o.flags = int(self.flags)
        return o


def torch_allocator(device: int):
    """(alloc, free) callbacks of an hg_allocator backed by the torch caching
    allocator on `device`: workspace and scene memory of the library then
    comes from (and returns to) the same pool as the caller's tensors.  The
    library frees a buffer only after the work that used it has finished
    (it synchronises first), so a block may be reused on any stream."""
    import torch

    def alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:  # out of memory (or any failure): the library reports HG_ERR_OOM
            return None

    def free(ptr, nbytes, stream, user):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass
    return alloc, free


class Context:
    """hg_ctx on one CUDA device.  allocator: "torch" (default) backs the
    library's device memory with the torch caching allocator; "cuda" lets
    the library call cudaMalloc / cudaFree; or an (alloc, free) pair of
    Python callables with the hg_allocator signatures (alloc(bytes, stream,
    user) -> device address or None; free(ptr, bytes, stream, user))."""

    def __init__(self, device: int = 0, allocator="torch"):
        self.lib = load()
        h = C.c_void_p()
        self._alloc = None
        if allocator == "torch":
            allocator = torch_allocator(device)
        if allocator == "cuda" or allocator is None:
            check(self.lib.hg_ctx_create(device, None, C.byref(h)))
        else:
            fa, ff = allocator
            # the callbacks must outlive the context: kept on self
            self._alloc = AllocatorC(ALLOC_FN(fa), FREE_FN(ff), None)
            check(self.lib.hg_ctx_create(device, C.byref(self._alloc), C.byref(h)))
        self.h = h
        self.device = device

    def set_wait_limits(self, wait_polls: int = -1, chain_polls: int = -1):
        """hg_ctx_set_wait_limits: polls before a bounded device wait gives
        up (mbarrier / look-back) and before a batch renders unchained; 0
        gives up at once, -1 restores the default."""
        check(self.lib.hg_ctx_set_wait_limits(self.h, int(wait_polls), int(chain_polls)))

    def close(self):
        if self.h:
            self.lib.hg_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GpuScene:
    """Device-resident scene (hg_create_scene).  Arrays are torch CUDA tensors
    (float32, contiguous; SH in the storage type sh_storage, converted with
    round-to-nearest-even when given in another type); borrow=True keeps
    references instead of copying.  order=ORDER_SPATIAL stores the gaussians
    in hg_spatial_order (owned copies only); order() returns the stored
    order as the caller's indices."""

    def __init__(self, ctx: Context, means, log_scales, quats, opacity_logits, sh, sh_degree: int,
                 borrow: bool = False, sh_storage: int = SH_F32, order: int = ORDER_INPUT):
        import torch
        dev = torch.device("cuda", ctx.device)

        def t(x, dtype=torch.float32):
            x = torch.as_tensor(x, device=dev)
            if x.dtype != dtype:
                x = x.to(torch.float32).to(dtype)
            return x.contiguous()
        sh_t = {SH_F32: torch.float32, SH_F16: torch.float16, SH_BF16: torch.bfloat16,
                SH_CODEC32: torch.float32}[sh_storage]
        self.tensors = [t(means), t(log_scales), t(quats), t(opacity_logits), t(sh, sh_t)]
        n = self.tensors[0].shape[0]
        d = SceneDesc(n, sh_degree, int(borrow), *[x.data_ptr() for x in self.tensors], sh_storage, order)
        h = C.c_void_p()
        torch.cuda.synchronize(dev)
        check(ctx.lib.hg_create_scene(ctx.h, C.byref(d), C.byref(h)))
        self.h, self.ctx, self.n, self.sh_degree, self.borrow = h, ctx, n, sh_degree, borrow
        self.sh_storage = sh_storage
        if not borrow:
            self.tensors = None

    def sh_codec(self):
        """Packed SH of a SH_CODEC32 scene: (scales [16][3], codes [n][8])."""
        scales = np.zeros((16, 3), np.float32)
        codes = np.zeros((self.n, 8), np.uint32)
        check(self.ctx.lib.hg_scene_sh_codec(self.h, scales.ctypes.data_as(C.c_void_p),
                                             codes.ctypes.data_as(C.c_void_p)))
        return scales, codes

    def order(self):
        """Stored order (hg_scene_order): int32 [n], the caller's index of
        each stored gaussian."""
        perm = np.zeros(self.n, np.int32)
        check(self.ctx.lib.hg_scene_order(self.h, perm.ctypes.data_as(C.c_void_p)))
        return perm

    @classmethod
    def from_scene(cls, ctx: Context, scene, borrow: bool = False, sh_storage: int = SH_F32,
                   order: int = ORDER_INPUT):
        return cls(ctx, scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh,
                   scene.sh_degree, borrow, sh_storage, order)

    def close(self):
        if self.h:
            self.ctx.lib.hg_destroy_scene(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """hg_state: a frame workspace plus what the last frame saved."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        self.h = C.c_void_p()

    def stats(self) -> dict:
        s = FrameStats()
        check(self.ctx.lib.hg_render_stats(self.h, C.byref(s)))
        return s.as_dict()

    def read(self, which: int, dtype=np.uint32) -> np.ndarray:
        need = C.c_size_t()
        check(self.ctx.lib.hg_state_read(self.h, which, None, 0, C.byref(need)))
        out = np.empty(need.value // np.dtype(dtype).itemsize, dtype)
        check(self.ctx.lib.hg_state_read(self.h, which, out.ctypes.data_as(C.c_void_p), out.nbytes,
                                         C.byref(need)))
        return out

    def sync(self) -> int:
        return self.ctx.lib.hg_state_sync(self.h)

    def close(self):
        if self.h:
            self.ctx.lib.hg_state_free(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _out_tensors(cams, device, out_rgb=None, out_T=None, with_T=True):
    import torch
    pix = sum(int(c.width) * int(c.height) for c in cams)
    if out_rgb is None:
        out_rgb = torch.empty(pix * 3, dtype=torch.float32, device=device)
    if out_T is None and with_T:
        out_T = torch.empty(pix, dtype=torch.float32, device=device)
    return out_rgb, out_T


class Graph:
    """A captured multi-view frame (hg_graph_*): replay with new poses of the
    same resolutions."""

    def __init__(self, scene: GpuScene, cams, opts: Options, out_rgb, out_T, state: State, stream):
        self.lib = scene.ctx.lib
        if not state.h:
            # the state's workspace is created by a first synchronous render
            render(scene, cams, Options(**{**opts.__dict__, "flags": 0}), state=state, stream=stream,
                   out_rgb=out_rgb, out_T=out_T)
        cam_arr = cameras_array(cams)
        o = opts.struct()
        h = C.c_void_p()
        check(self.lib.hg_graph_create(scene.h, cam_arr, len(cams), C.byref(o), C.c_void_p(out_rgb.data_ptr()),
                                       C.c_void_p(out_T.data_ptr()) if out_T is not None else None, state.h,
                                       C.c_void_p(stream.cuda_stream), C.byref(h)))
        self.h, self.state, self.scene, self.stream, self.n_views = h, state, scene, stream, len(cams)
        self.kernels = int(self.lib.hg_graph_kernels(h))

    def set_cameras(self, cams):
        check(self.lib.hg_graph_set_cameras(self.h, cameras_array(cams), len(cams)))

    def launch(self, stream=None):
        s = self.stream if stream is None else stream
        check(self.lib.hg_graph_launch(self.h, C.c_void_p(s.cuda_stream)))

    def sync(self):
        check(self.lib.hg_graph_sync(self.h))

    def close(self):
        if self.h:
            self.lib.hg_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_sort_args(seg_off, keys, vals, keys_out, vals_out, require_cuda: bool = True):
    """Raise ValueError unless the five tensors of segmented_sort_noalloc fit
    the entry point: contiguous 4-byte integer tensors (seg_off int32 or
    uint32 with at least 2 entries, the pairs int32 / uint32 / float32 bit
    patterns), keys, vals, keys_out and vals_out of the same length, and, with
    require_cuda, all on the current CUDA device."""
    import torch
    named = (("seg_off", seg_off), ("keys", keys), ("vals", vals), ("keys_out", keys_out), ("vals_out", vals_out))
    for name, t in named:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if require_cuda:
            if not t.is_cuda or t.device.index != torch.cuda.current_device():
                raise ValueError(f"{name} must be a CUDA tensor on the current device")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if seg_off.dtype not in (torch.int32, torch.uint32):
        raise ValueError("seg_off must be int32 or uint32")
    if seg_off.numel() < 2:
        raise ValueError("seg_off needs at least 2 entries (one segment)")
    for name, t in named[1:]:
        if t.dtype not in (torch.int32, torch.uint32, torch.float32):
            raise ValueError(f"{name} must have a 4-byte dtype (int32, uint32 or float32)")
        if t.numel() != keys.numel():
            raise ValueError(f"{name} has {t.numel()} elements, keys has {keys.numel()}")


def segmented_sort_noalloc(seg_off, keys, vals, keys_out, vals_out, stream=None) -> int:
    """hg_segmented_sort_noalloc on device int32/uint32 tensors; returns the
    hg_status (no exception) so callers can inspect rejections.  Malformed
    tensors raise ValueError before the library is called."""
    check_sort_args(seg_off, keys, vals, keys_out, vals_out)
    return int(load().hg_segmented_sort_noalloc(C.c_void_p(seg_off.data_ptr()), int(seg_off.numel()) - 1,
                                                int(keys.numel()), C.c_void_p(keys.data_ptr()),
                                                C.c_void_p(vals.data_ptr()), C.c_void_p(keys_out.data_ptr()),
                                                C.c_void_p(vals_out.data_ptr()), _stream_ptr(stream)))


def render_backward(state: State, scene: GpuScene, dl_drgb, stream=None, out=None):
    """hg_render_backward for the frame saved in `state`: returns device
    tensors (d_means, d_log_scales, d_quats, d_opacity_logits, d_sh), written
    into `out` when given."""
    import torch
    dev = torch.device("cuda", scene.ctx.device)
    n, k = scene.n, (scene.sh_degree + 1) ** 2
    outs = out if out is not None else [torch.empty((n, 3), device=dev), torch.empty((n, 3), device=dev),
                                        torch.empty((n, 4), device=dev), torch.empty((n,), device=dev),
                                        torch.empty((n, k, 3), device=dev)]
    g = dl_drgb.contiguous().to(torch.float32)
    check(scene.ctx.lib.hg_render_backward(state.h, C.c_void_p(g.data_ptr()),
                                           *[C.c_void_p(o.data_ptr()) for o in outs], _stream_ptr(stream)))
    return tuple(outs)


def spatial_order(ctx: Context, means, stream=None):
    """hg_spatial_order: int32 CUDA tensor [n], the indices of the gaussians
    (means: float32 CUDA [n][3]) in ascending Morton code, ties by index."""
    import torch
    means = torch.as_tensor(means, device=torch.device("cuda", ctx.device)).to(torch.float32).contiguous()
    n = means.shape[0]
    perm = torch.empty(n, dtype=torch.int32, device=means.device)
    check(ctx.lib.hg_spatial_order(ctx.h, C.c_void_p(means.data_ptr()), n, C.c_void_p(perm.data_ptr()),
                                   _stream_ptr(stream)))
    return perm


def l2_loss(ctx: Context, rgb, target, dl_drgb=None, loss=None, stream=None):
    """hg_l2_loss: returns (loss as a device float64 tensor of one element,
    dL/d rgb as a device float32 tensor)."""
    import torch
    dev = torch.device("cuda", ctx.device)
    rgb = rgb.contiguous()
    target = target.contiguous()
    if dl_drgb is None:
        dl_drgb = torch.empty_like(rgb)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float64, device=dev)
    check(ctx.lib.hg_l2_loss(ctx.h, C.c_void_p(rgb.data_ptr()), C.c_void_p(target.data_ptr()), rgb.numel(),
                             C.c_void_p(dl_drgb.data_ptr()), C.c_void_p(loss.data_ptr()), _stream_ptr(stream)))
    return loss, dl_drgb


def adam_step(scene: GpuScene, grads, m, v, step: int, lr, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """hg_adam_step on the scene's parameter arrays (five groups: means,
    log_scales, quats, opacity_logits, sh); lr is a number or five numbers."""
    lrs = list(lr) if hasattr(lr, "__len__") else [lr] * 5
    o = AdamOpts((C.c_float * 5)(*lrs), beta1, beta2, eps, step)
    arr = C.c_void_p * 5
    check(scene.ctx.lib.hg_adam_step(scene.h, arr(*[x.data_ptr() for x in grads]), arr(*[x.data_ptr() for x in m]),
                                     arr(*[x.data_ptr() for x in v]), C.byref(o), _stream_ptr(stream)))


class Trainer:
    """Densification-free optimisation of a scene against target images
    (Sec. 6): per step hg_render (saving for the backward), hg_l2_loss,
    hg_render_backward and hg_adam_step, all on one stream.  The parameters
    are the caller's tensors (a borrowed scene), updated in place."""

    # 3DGS-style learning rates: means, log_scales, quats, opacity logits, SH
    DEFAULT_LR = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3)

    def __init__(self, ctx: Context, params, sh_degree: int, cams, target, opts: Options | None = None,
                 lr=DEFAULT_LR, stream=None):
        import torch
        self.ctx, self.cams, self.stream = ctx, list(cams), stream
        self.params = [p.contiguous() for p in params]
        self.scene = GpuScene(ctx, *self.params, sh_degree=sh_degree, borrow=True)
        # default: macro 4x4, B_r = 512, ellipse binning, the fastest training
        # step measured on the 1M scene (the backward keeps per-gaussian
        # gradient sums of the unit in shared memory, so smaller batches fit
        # more CTAs per SM than the forward's best B_r = 1024)
        base = opts or Options(macro_w=4, macro_h=4, batch_cap=512, bin_test=BIN_ELLIPSE)
        self.opts = Options(**{**base.__dict__, "save_for_backward": True})
        self.target = target.contiguous()
        self.state = State(ctx)
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.lr, self.t = lr, 0
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.target.device)
        self.dl = torch.empty_like(self.target)
        self.grads = [torch.empty_like(p) for p in self.params]

    def step(self):
        """One optimisation step; returns the loss of the rendered frame as a
        device tensor (reading it synchronises)."""
        rgb, _ = render(self.scene, self.cams, self.opts, state=self.state, stream=self.stream, with_T=False)
        l2_loss(self.ctx, rgb, self.target, self.dl, self.loss, stream=self.stream)
        render_backward(self.state, self.scene, self.dl, stream=self.stream, out=self.grads)
        self.t += 1
        adam_step(self.scene, self.grads, self.m, self.v, self.t, self.lr, stream=self.stream)
        return self.loss

    def close(self):
        self.state.close()
        self.scene.close()


class _RenderFn:
    """torch.autograd.Function wrapping hg_render / hg_render_backward."""
    fn = None

    @classmethod
    def get(cls):
        if cls.fn is None:
            import torch

            class RenderFunction(torch.autograd.Function):
                @staticmethod
                def forward(ctx, means, log_scales, quats, opacity_logits, sh, gctx, cams, opts, sh_degree):
                    scene = GpuScene(gctx, means.detach(), log_scales.detach(), quats.detach(),
                                     opacity_logits.detach(), sh.detach(), sh_degree, borrow=True)
                    state = State(gctx)
                    o = Options(**{**opts.__dict__, "save_for_backward": True, "path": PATH_HIGS})
                    rgb, _ = render(scene, cams, o, state=state, with_T=False)
                    ctx.hg = (scene, state)
                    return rgb

                @staticmethod
                def backward(ctx, grad_rgb):
                    scene, state = ctx.hg
                    grads = render_backward(state, scene, grad_rgb)
                    return (*grads, None, None, None, None)

            cls.fn = RenderFunction
        return cls.fn


def render_differentiable(gctx: Context, means, log_scales, quats, opacity_logits, sh, sh_degree: int, cams,
                          opts: Options | None = None):
    """Differentiable render of views `cams`: packed rgb [sum_v H_v W_v * 3]
    whose gradient flows to the five scene tensors (float32 CUDA)."""
    return _RenderFn.get().apply(means, log_scales, quats, opacity_logits, sh, gctx, cams, opts or Options(),
                                 sh_degree)


def autotune(scene: GpuScene, cams, base: Options | None = None, iters: int = 3, cache_path: str | None = None,
             stream=None):
    """hg_autotune: returns (best Options, [(macro_w, macro_h, batch_cap, ms)])."""
    base = base or Options()
    best = RenderOpts()
    res = (TuneResult * 16)()
    nres = C.c_int()
    check(scene.ctx.lib.hg_autotune(scene.h, cameras_array(cams), len(cams), C.byref(base.struct()), iters,
                                    cache_path.encode() if cache_path else None, C.byref(best), res, 16,
                                    C.byref(nres), _stream_ptr(stream)))
    opts = Options(path=best.path, macro_w=best.macro_w, macro_h=best.macro_h, batch_cap=best.batch_cap,
                   bg=tuple(best.bg), save_for_backward=bool(best.save_for_backward), flags=best.flags)
    return opts, [(r.macro_w, r.macro_h, r.batch_cap, r.ms) for r in res[:nres.value]]


class Server:
    """Continuous-batching render server (hg_serve_*)."""

    def __init__(self, ctx: Context, max_inflight: int = 4, max_views_per_launch: int = 8, mem_budget_bytes: int = 0,
                 batch_window_us: int = 0, opts: Options | None = None, presize=(0, 0)):
        """presize=(W, H): size every slot, when a scene is added, for
        max_views_per_launch views at W x H (no workspace growth while
        serving up to that size)."""
        self.ctx, self.lib = ctx, ctx.lib
        cfg = ServeConfig(max_inflight, max_views_per_launch, mem_budget_bytes, batch_window_us, int(presize[0]),
                          int(presize[1]), 0, (opts or Options()).struct())
        h = C.c_void_p()
        check(self.lib.hg_serve_create(ctx.h, C.byref(cfg), C.byref(h)))
        self.h = h
        self.scenes = []

    def add_scene(self, scene: GpuScene) -> int:
        sid = C.c_int()
        check(self.lib.hg_serve_add_scene(self.h, scene.h, C.byref(sid)))
        self.scenes.append(scene)
        return sid.value

    def submit(self, scene_id: int, cam, out, on_host: bool = False) -> int:
        """Non-blocking; `out` is a float32 tensor of H*W*3 (CUDA, or pinned CPU)."""
        rid = C.c_uint64()
        check(self.lib.hg_serve_submit(self.h, scene_id, C.byref(camera_struct(cam)), C.c_void_p(out.data_ptr()),
                                       int(on_host), C.byref(rid)))
        return rid.value

    def submit_status(self, scene_id: int, cam, out, on_host: bool = False):
        rid = C.c_uint64()
        st = self.lib.hg_serve_submit(self.h, scene_id, C.byref(camera_struct(cam)), C.c_void_p(out.data_ptr()),
                                      int(on_host), C.byref(rid))
        return st, rid.value

    def poll(self, rid: int) -> bool:
        done = C.c_int()
        st = self.lib.hg_serve_poll(self.h, rid, C.byref(done))
        if done.value:
            check(st)
        return bool(done.value)

    def wait(self, rid: int, timeout_ms: int = -1) -> int:
        return int(self.lib.hg_serve_wait(self.h, rid, timeout_ms))

    def cancel(self, rid: int) -> int:
        return int(self.lib.hg_serve_cancel(self.h, rid))

    def stats(self) -> dict:
        s = ServeStats()
        check(self.lib.hg_serve_stats(self.h, C.byref(s)))
        return s.as_dict()

    def reset_stats(self):
        check(self.lib.hg_serve_reset_stats(self.h))

    def close(self):
        if self.h:
            self.lib.hg_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    return int(load().hg_kernel_launches())


def split_views(flat, cams, channels):
    out, o = [], 0
    for c in cams:
        k = int(c.width) * int(c.height)
        out.append(flat[o * channels:(o + k) * channels].view(int(c.height), int(c.width), *([channels] if channels > 1 else [])))
        o += k
    return out


def render(scene: GpuScene, cams, opts: Options | None = None, state: State | None = None, stream=None,
           out_rgb=None, out_T=None, with_T=True):
    """Render `cams` (list of scenes.Camera) of `scene`.  Returns the packed
    (rgb, T) device tensors (views back to back)."""
    import torch
    opts = opts or Options()
    dev = torch.device("cuda", scene.ctx.device)
    out_rgb, out_T = _out_tensors(cams, dev, out_rgb, out_T, with_T)
    cam_arr = cameras_array(cams)
    o = opts.struct()
    sp = C.byref(state.h) if state is not None else None
    check(scene.ctx.lib.hg_render(scene.h, cam_arr, len(cams), C.byref(o), C.c_void_p(out_rgb.data_ptr()),
                                  C.c_void_p(out_T.data_ptr()) if out_T is not None else None, sp,
                                  _stream_ptr(stream)))
    return out_rgb, out_T


def render_splats(ctx: Context, splats, n: int, cams, opts: Options | None = None, state: State | None = None,
                  stream=None):
    """Render precomputed splats (device uint8 tensor of [V][n] hg_splat)."""
    import torch
    opts = opts or Options()
    dev = torch.device("cuda", ctx.device)
    out_rgb, out_T = _out_tensors(cams, dev)
    cam_arr = cameras_array(cams)
    o = opts.struct()
    sp = C.byref(state.h) if state is not None else None
    check(ctx.lib.hg_render_splats(ctx.h, C.c_void_p(splats.data_ptr()), n, cam_arr, len(cams), C.byref(o),
                                   C.c_void_p(out_rgb.data_ptr()), C.c_void_p(out_T.data_ptr()), sp,
                                   _stream_ptr(stream)))
    return out_rgb, out_T


def splats_to_device(rec: np.ndarray, device=0):
    """numpy structured array (SPLAT_DTYPE) -> device byte tensor."""
    import torch
    assert rec.dtype == SPLAT_DTYPE
    return torch.from_numpy(rec.view(np.uint8).copy()).to(torch.device("cuda", device))


def version() -> str:
    return load().hg_version().decode()
