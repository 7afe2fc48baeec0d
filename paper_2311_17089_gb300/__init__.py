"""Python binding of libmsgs (include/msgs.h): multi-scale selective
Gaussian splatting on one GPU.

Argument marshalling only: every step of the rendering path runs in the
CUDA kernels of libmsgs.so.  PyTorch provides device memory and streams.
The functions `ms_*` mirror the C entry points one to one and raise
`MsError` on a non-zero status.  `DeviceScene` and `Renderer` hold the
torch-allocated buffers a frame needs and chain the calls; `render_views`
renders several frames of one scene from one `ms_project_views` pass.

There is no CPU fallback: if libmsgs.so cannot be built or loaded, or no
CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
# MSGS_DEBUG=1 loads the debug build (index checks reported as MS_ERR_BOUNDS)
DEBUG = os.environ.get("MSGS_DEBUG", "0") == "1"
LIB_PATH = os.path.join(_HERE, "libmsgs_debug.so" if DEBUG else "libmsgs.so")

MS_OK, MS_ERR_INVALID_ARG, MS_ERR_CAPACITY, MS_ERR_CUDA, MS_ERR_TIMEOUT = 0, 1, 2, 3, 4
MS_ERR_NO_DEVICE, MS_PENDING, MS_ERR_OOM, MS_ERR_BOUNDS = 5, 6, 7, 8
MS_SELECTIVE, MS_ALL_LEVELS, MS_FILTER_SMALL = 0, 1, 2
MODES = {"selective": MS_SELECTIVE, "all_levels": MS_ALL_LEVELS,
         "filter_small": MS_FILTER_SMALL}
MS_RASTER_AUTO, MS_RASTER_TILE, MS_RASTER_LIST = 0, 1, 2
MS_RASTER_GROUP8, MS_RASTER_GROUP16, MS_RASTER_GROUP32 = 3, 4, 5
STRATEGIES = {"auto": MS_RASTER_AUTO, "tile": MS_RASTER_TILE, "list": MS_RASTER_LIST,
              "group8": MS_RASTER_GROUP8, "group16": MS_RASTER_GROUP16,
              "group32": MS_RASTER_GROUP32}
MS_STATS_WORDS = 1040
MS_BWD_ACCUMULATE = 1
MS_BWD_RASTER_PASS = 2
MS_BWD_PROJECT_PASS = 4
MS_MAX_BWD_VIEWS = 8
REC_FLOATS = 12

P = ctypes.c_void_p


class MsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"msgs error {code}: {msg}")
        self.code = code


class ms_scene_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_levels", ctypes.c_int32),
                ("sh_degree", ctypes.c_int32), ("mean", P), ("log_scale", P),
                ("quat", P), ("opacity", P), ("color", P), ("level", P),
                ("s_max", P), ("s_min", P), ("scale", P), ("lnop", P)]


class ms_camera_t(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("campos", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_plane", ctypes.c_float),
                ("bg", ctypes.c_float * 3)]


class ms_proj_t(ctypes.Structure):
    _fields_ = [("rec", P), ("rect", P), ("n_tiles", P), ("depth", P),
                ("cover", P), ("mask", P), ("stats", P), ("n", ctypes.c_int64)]


class ms_grads_t(ctypes.Structure):
    _fields_ = [("dmean", P), ("dlog_scale", P), ("dquat", P), ("dopacity", P),
                ("dcolor", P)]


class ms_bins_t(ctypes.Structure):
    _fields_ = [("gauss_idx", P), ("ranges", P), ("counts", P),
                ("dup_capacity", ctypes.c_int64)]


class ms_bwd_view_t(ctypes.Structure):
    _fields_ = [("cam", ms_camera_t), ("proj", ctypes.POINTER(ms_proj_t)),
                ("bins", ctypes.POINTER(ms_bins_t)), ("image", P), ("n_contrib", P),
                ("raster_ws", P), ("raster_ws_bytes", ctypes.c_size_t), ("dl_dimage", P)]


class ms_serve_cfg_t(ctypes.Structure):
    _fields_ = [("max_gaussians", ctypes.c_int64), ("max_width", ctypes.c_int32),
                ("max_height", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_size_t),
                ("initial_capacity", ctypes.c_int64), ("device", ctypes.c_int32),
                ("max_batch_views", ctypes.c_int32)]


class ms_request_t(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_int32), ("mode", ctypes.c_int32), ("cam", ms_camera_t),
                ("image_dev", P), ("image_host", P)]


class ms_result_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("retries", ctypes.c_int32),
                ("duplicates", ctypes.c_int64), ("capacity", ctypes.c_int64),
                ("bytes", ctypes.c_size_t), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class ms_serve_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("retries", ctypes.c_int64),
                ("queued", ctypes.c_int32), ("inflight", ctypes.c_int32),
                ("peak_inflight", ctypes.c_int32), ("scenes", ctypes.c_int32),
                ("arena_bytes", ctypes.c_size_t), ("arena_used", ctypes.c_size_t),
                ("arena_peak", ctypes.c_size_t), ("renders", ctypes.c_int64),
                ("issue_seconds", ctypes.c_double), ("proj_passes", ctypes.c_int64),
                ("proj_seconds", ctypes.c_double)]


# (name, restype, argtypes) of every entry point declared in include/msgs.h
_SIGNATURES = [
    ("ms_last_error", ctypes.c_char_p, []),
    ("ms_version", ctypes.c_int, []),
    ("ms_scene_prepare", ctypes.c_int, [ctypes.POINTER(ms_scene_t), P]),
    ("ms_project", ctypes.c_int, [ctypes.POINTER(ms_scene_t), ctypes.POINTER(ms_camera_t),
                                  ctypes.c_int, ctypes.POINTER(ms_proj_t), P]),
    ("ms_project_views", ctypes.c_int, [ctypes.POINTER(ms_scene_t), ctypes.POINTER(ms_camera_t),
                                        ctypes.c_int32, ctypes.c_int, ctypes.POINTER(ms_proj_t),
                                        P]),
    ("ms_project_views_update", ctypes.c_int, [ctypes.POINTER(ms_scene_t),
                                               ctypes.POINTER(ms_camera_t), ctypes.c_int32,
                                               ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(ms_proj_t), P]),
    ("ms_project_views_union", ctypes.c_int, [ctypes.POINTER(ms_scene_t),
                                              ctypes.POINTER(ms_camera_t), ctypes.c_int32,
                                              ctypes.c_int, ctypes.POINTER(ms_proj_t),
                                              ctypes.c_uint32, P, P, P]),
    ("ms_sort_depth_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64]),
    ("ms_sort_depth", ctypes.c_int, [ctypes.POINTER(ms_proj_t), ctypes.c_int64, P, P,
                                     ctypes.c_size_t, P]),
    ("ms_split_order_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64]),
    ("ms_split_order", ctypes.c_int, [ctypes.POINTER(ms_proj_t), ctypes.c_int64, P,
                                      ctypes.c_int32, P, P, P, ctypes.c_size_t, P]),
    ("ms_bin_ordered", ctypes.c_int, [ctypes.POINTER(ms_proj_t), ctypes.c_int64,
                                      ctypes.POINTER(ms_camera_t), ctypes.POINTER(ms_bins_t),
                                      P, P, P, ctypes.c_size_t, P]),
    ("ms_select", ctypes.c_int, [ctypes.POINTER(ms_scene_t), P, ctypes.c_int, P, P]),
    ("ms_update_range", ctypes.c_int, [ctypes.POINTER(ms_scene_t),
                                       ctypes.POINTER(ms_camera_t), ctypes.c_int32, P]),
    ("ms_bin_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.c_int64]),
    ("ms_bin", ctypes.c_int, [ctypes.POINTER(ms_proj_t), ctypes.c_int64,
                              ctypes.POINTER(ms_camera_t), ctypes.POINTER(ms_bins_t),
                              P, ctypes.c_size_t, P]),
    ("ms_bin_noalloc", ctypes.c_int, [ctypes.POINTER(ms_proj_t), ctypes.c_int64,
                                      ctypes.POINTER(ms_camera_t), ctypes.POINTER(ms_bins_t),
                                      P]),
    ("ms_bin_counts", ctypes.c_int, [ctypes.POINTER(ms_bins_t),
                                     ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int64), P]),
    ("ms_raster_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64]),
    ("ms_raster_bwd_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64]),
    ("ms_raster_bwd", ctypes.c_int, [ctypes.POINTER(ms_scene_t), ctypes.POINTER(ms_camera_t),
                                     ctypes.POINTER(ms_proj_t), ctypes.POINTER(ms_bins_t),
                                     P, P, P, ctypes.c_size_t, P, ctypes.POINTER(ms_grads_t),
                                     ctypes.c_uint32, P, ctypes.c_size_t, P]),
    ("ms_raster_bwd_views_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int32]),
    ("ms_raster_bwd_views", ctypes.c_int, [ctypes.POINTER(ms_scene_t),
                                           ctypes.POINTER(ms_bwd_view_t), ctypes.c_int32,
                                           ctypes.POINTER(ms_grads_t), ctypes.c_uint32, P,
                                           ctypes.c_size_t, P]),
    ("ms_l1_loss_grad", ctypes.c_int, [P, P, ctypes.c_int64, ctypes.c_float, P, P, P]),
    ("ms_raster", ctypes.c_int, [ctypes.POINTER(ms_proj_t), ctypes.POINTER(ms_bins_t),
                                 ctypes.POINTER(ms_camera_t), P, P, P, P, P,
                                 ctypes.c_size_t, P]),
    ("ms_raster_ex", ctypes.c_int, [ctypes.POINTER(ms_proj_t), ctypes.POINTER(ms_bins_t),
                                    ctypes.POINTER(ms_camera_t), P, P, P, P, P,
                                    ctypes.c_size_t, ctypes.c_int, P]),
    ("ms_raster_ex2", ctypes.c_int, [ctypes.POINTER(ms_proj_t), ctypes.POINTER(ms_bins_t),
                                     ctypes.POINTER(ms_camera_t), P, P, P, P, P,
                                     ctypes.c_size_t, ctypes.c_int, ctypes.c_int32, P]),
    ("ms_aggregate_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64]),
    ("ms_aggregate", ctypes.c_int, [ctypes.POINTER(ms_scene_t), ctypes.POINTER(ms_camera_t),
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                    ctypes.POINTER(ms_scene_t), ctypes.c_int64, P, P,
                                    ctypes.c_size_t, P]),
    ("ms_serve_clock", ctypes.c_double, []),
    ("ms_serve_create", ctypes.c_int, [ctypes.POINTER(ms_serve_cfg_t), ctypes.POINTER(P)]),
    ("ms_serve_add_scene", ctypes.c_int, [P, ctypes.POINTER(ms_scene_t),
                                          ctypes.POINTER(ctypes.c_int32)]),
    ("ms_serve_submit", ctypes.c_int, [P, ctypes.POINTER(ms_request_t),
                                       ctypes.POINTER(ctypes.c_uint64)]),
    ("ms_serve_poll", ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(ms_result_t)]),
    ("ms_serve_wait", ctypes.c_int, [P, ctypes.c_uint64, ctypes.c_double,
                                     ctypes.POINTER(ms_result_t)]),
    ("ms_serve_stats", ctypes.c_int, [P, ctypes.POINTER(ms_serve_stats_t)]),
    ("ms_serve_destroy", ctypes.c_int, [P]),
    ("ms_debug_set_spin_limit", ctypes.c_int, [ctypes.c_uint32]),
    ("ms_alu_probe", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]),
    ("ms_alu_probe_ops", ctypes.c_double, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
]

_lib = None


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force, debug=DEBUG)


def lib():
    """Load libmsgs.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        from . import _build
        if not _build.up_to_date(DEBUG):
            _build.build(debug=DEBUG)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != MS_OK:
        raise MsError(rc, lib().ms_last_error().decode())


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(stream=None) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def camera_struct(cam: inputs.Camera) -> ms_camera_t:
    c = ms_camera_t()
    c.R[:] = [float(v) for v in np.asarray(cam.R, np.float32).reshape(9)]
    c.t[:] = [float(v) for v in np.asarray(cam.t, np.float32)]
    c.campos[:] = [float(v) for v in np.asarray(cam.campos, np.float32)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = cam.width, cam.height
    c.near_plane = cam.near
    c.bg[:] = [float(v) for v in np.asarray(cam.bg, np.float32)]
    return c


# ------------------------------------------------ one-to-one entry points

def ms_version() -> int:
    return lib().ms_version()


def ms_scene_prepare(scene: ms_scene_t, stream=None):
    _check(lib().ms_scene_prepare(ctypes.byref(scene), P(_stream(stream))))


def ms_project(scene: ms_scene_t, cam: ms_camera_t, mode: int, out: ms_proj_t, stream=None):
    _check(lib().ms_project(ctypes.byref(scene), ctypes.byref(cam), int(mode),
                            ctypes.byref(out), P(_stream(stream))))


MS_MAX_PROJ_VIEWS = 8


def ms_project_views(scene: ms_scene_t, cams, mode: int, outs, stream=None):
    """ms_project for len(cams) <= MS_MAX_PROJ_VIEWS cameras in one pass;
    outs[v] (an ms_proj_t) receives view v's outputs."""
    n = len(cams)
    if len(outs) != n:
        raise MsError(MS_ERR_INVALID_ARG, "one ms_proj_t per camera")
    ca = (ms_camera_t * max(n, 1))(*cams)
    oa = (ms_proj_t * max(n, 1))(*outs)
    _check(lib().ms_project_views(ctypes.byref(scene), ca, n, int(mode), oa,
                                  P(_stream(stream))))


def ms_project_views_update(scene: ms_scene_t, cams, mode: int, update_levels, outs,
                            stream=None):
    """ms_project_views with UpdateRange (Eq. 5) fused: view v updates the
    coverage ranges of level update_levels[v] (0: none) after its
    selection, in view order."""
    n = len(cams)
    if len(outs) != n or len(update_levels) != n:
        raise MsError(MS_ERR_INVALID_ARG, "one ms_proj_t and one update level per camera")
    ca = (ms_camera_t * max(n, 1))(*cams)
    oa = (ms_proj_t * max(n, 1))(*outs)
    la = (ctypes.c_int32 * max(n, 1))(*[int(x) for x in update_levels])
    _check(lib().ms_project_views_update(ctypes.byref(scene), ca, n, int(mode), la, oa,
                                         P(_stream(stream))))


def ms_project_views_union(scene: ms_scene_t, cams, mode: int, outs, union_views: int,
                           union_flags_ptr: int, union_stats_ptr: int, stream=None):
    """ms_project_views, also writing the union of the listed Gaussians of
    the views in the bit mask union_views (one pose) for ms_sort_depth."""
    n = len(cams)
    if len(outs) != n:
        raise MsError(MS_ERR_INVALID_ARG, "one ms_proj_t per camera")
    ca = (ms_camera_t * max(n, 1))(*cams)
    oa = (ms_proj_t * max(n, 1))(*outs)
    _check(lib().ms_project_views_union(ctypes.byref(scene), ca, n, int(mode), oa,
                                        int(union_views), P(union_flags_ptr),
                                        P(union_stats_ptr), P(_stream(stream))))


def ms_sort_depth_workspace_bytes(n: int) -> int:
    return int(lib().ms_sort_depth_workspace_bytes(int(n)))


def ms_sort_depth(proj: ms_proj_t, n: int, order_ptr: int, ws_ptr: int, ws_bytes: int,
                  stream=None):
    _check(lib().ms_sort_depth(ctypes.byref(proj), int(n), P(order_ptr), P(ws_ptr), ws_bytes,
                               P(_stream(stream))))


def ms_split_order_workspace_bytes(n: int) -> int:
    return int(lib().ms_split_order_workspace_bytes(int(n)))


def ms_split_order(union_proj: ms_proj_t, n: int, order_ptr: int, order_ptrs, stats_ptrs,
                   ws_ptr: int, ws_bytes: int, stream=None):
    """The union's depth order restricted to each view (orders[v], with the
    view's count and the union's status in view_stats[v])."""
    k = len(order_ptrs)
    if len(stats_ptrs) != k:
        raise MsError(MS_ERR_INVALID_ARG, "one stats array per order")
    oa = (ctypes.c_void_p * max(k, 1))(*order_ptrs)
    sa = (ctypes.c_void_p * max(k, 1))(*stats_ptrs)
    _check(lib().ms_split_order(ctypes.byref(union_proj), int(n), P(order_ptr), k, oa, sa,
                                P(ws_ptr), ws_bytes, P(_stream(stream))))


def ms_bin_ordered(proj: ms_proj_t, n: int, cam: ms_camera_t, out: ms_bins_t, order_ptr: int,
                   order_stats_ptr: int, ws_ptr: int, ws_bytes: int, stream=None):
    _check(lib().ms_bin_ordered(ctypes.byref(proj), int(n), ctypes.byref(cam), ctypes.byref(out),
                                P(order_ptr), P(order_stats_ptr), P(ws_ptr), ws_bytes,
                                P(_stream(stream))))


def ms_select(scene: ms_scene_t, cover_ptr: int, mode: int, mask_ptr: int, stream=None):
    _check(lib().ms_select(ctypes.byref(scene), P(cover_ptr), int(mode), P(mask_ptr),
                           P(_stream(stream))))


def ms_update_range(scene: ms_scene_t, cam: ms_camera_t, level_r: int, stream=None):
    _check(lib().ms_update_range(ctypes.byref(scene), ctypes.byref(cam), int(level_r),
                                 P(_stream(stream))))


def ms_bin_workspace_bytes(n: int, tiles: int, dup_capacity: int) -> int:
    return int(lib().ms_bin_workspace_bytes(n, tiles, dup_capacity))


def ms_bin(proj: ms_proj_t, n: int, cam: ms_camera_t, out: ms_bins_t, ws_ptr: int,
           ws_bytes: int, stream=None):
    _check(lib().ms_bin(ctypes.byref(proj), int(n), ctypes.byref(cam), ctypes.byref(out),
                        P(ws_ptr), ws_bytes, P(_stream(stream))))


def ms_bin_noalloc(proj: ms_proj_t, n: int, cam: ms_camera_t, out: ms_bins_t, stream=None):
    """ms_bin with the library's static scratch array instead of a caller
    workspace, for callers that cannot allocate device memory."""
    _check(lib().ms_bin_noalloc(ctypes.byref(proj), int(n), ctypes.byref(cam),
                                ctypes.byref(out), P(_stream(stream))))


MS_PROBE_FFMA, MS_PROBE_FFMA2, MS_PROBE_EX2 = 0, 1, 2


def ms_debug_set_spin_limit(limit: int):
    """Test hook: ms_bin's look-back waits give up after `limit` polls
    (0: the default)."""
    _check(lib().ms_debug_set_spin_limit(int(limit)))


def ms_alu_probe(kind: int, blocks: int, iters: int, out_ptr: int, stream=None):
    """One throughput-probe launch (FFMA, packed FFMA2 or MUFU ex2)."""
    _check(lib().ms_alu_probe(int(kind), int(blocks), int(iters), P(out_ptr),
                              P(_stream(stream))))


def ms_alu_probe_ops(kind: int, blocks: int, iters: int) -> float:
    return float(lib().ms_alu_probe_ops(int(kind), int(blocks), int(iters)))


def ms_bin_counts(bins: ms_bins_t, stream=None):
    """(status, D needed, survivors); synchronises the stream."""
    d = ctypes.c_int64()
    s = ctypes.c_int64()
    rc = lib().ms_bin_counts(ctypes.byref(bins), ctypes.byref(d), ctypes.byref(s),
                             P(_stream(stream)))
    if rc not in (MS_OK, MS_ERR_CAPACITY):
        _check(rc)
    return rc, d.value, s.value


def ms_raster_workspace_bytes(tiles: int, dup_capacity: int) -> int:
    return int(lib().ms_raster_workspace_bytes(tiles, dup_capacity))


def ms_raster(proj: ms_proj_t, bins: ms_bins_t, cam: ms_camera_t, image_ptr: int,
              final_t_ptr: int, n_contrib_ptr: int, n_eval_ptr: int, ws_ptr: int,
              ws_bytes: int, stream=None):
    _check(lib().ms_raster(ctypes.byref(proj), ctypes.byref(bins), ctypes.byref(cam),
                           P(image_ptr), P(final_t_ptr), P(n_contrib_ptr), P(n_eval_ptr),
                           P(ws_ptr), ws_bytes, P(_stream(stream))))


def ms_raster_ex(proj: ms_proj_t, bins: ms_bins_t, cam: ms_camera_t, image_ptr: int,
                 final_t_ptr: int, n_contrib_ptr: int, n_eval_ptr: int, ws_ptr: int,
                 ws_bytes: int, strategy: int, stream=None):
    _check(lib().ms_raster_ex(ctypes.byref(proj), ctypes.byref(bins), ctypes.byref(cam),
                              P(image_ptr), P(final_t_ptr), P(n_contrib_ptr), P(n_eval_ptr),
                              P(ws_ptr), ws_bytes, int(strategy), P(_stream(stream))))


def ms_raster_ex2(proj: ms_proj_t, bins: ms_bins_t, cam: ms_camera_t, image_ptr: int,
                  final_t_ptr: int, n_contrib_ptr: int, n_eval_ptr: int, ws_ptr: int,
                  ws_bytes: int, strategy: int, max_ctas_per_sm: int, stream=None):
    _check(lib().ms_raster_ex2(ctypes.byref(proj), ctypes.byref(bins), ctypes.byref(cam),
                               P(image_ptr), P(final_t_ptr), P(n_contrib_ptr), P(n_eval_ptr),
                               P(ws_ptr), ws_bytes, int(strategy), int(max_ctas_per_sm),
                               P(_stream(stream))))


def ms_raster_bwd_workspace_bytes(n: int) -> int:
    return int(lib().ms_raster_bwd_workspace_bytes(n))


def ms_raster_bwd(scene: ms_scene_t, cam: ms_camera_t, proj: ms_proj_t, bins: ms_bins_t,
                  image_ptr: int, n_contrib_ptr: int, raster_ws_ptr: int, raster_ws_bytes: int,
                  dl_ptr: int, grads: ms_grads_t, flags: int, ws_ptr: int, ws_bytes: int,
                  stream=None):
    _check(lib().ms_raster_bwd(ctypes.byref(scene), ctypes.byref(cam), ctypes.byref(proj),
                               ctypes.byref(bins), P(image_ptr), P(n_contrib_ptr),
                               P(raster_ws_ptr), raster_ws_bytes, P(dl_ptr),
                               ctypes.byref(grads), int(flags), P(ws_ptr), ws_bytes,
                               P(_stream(stream))))


def ms_raster_bwd_views_workspace_bytes(n: int, n_views: int) -> int:
    return int(lib().ms_raster_bwd_views_workspace_bytes(n, n_views))


def bwd_view(cam: ms_camera_t, proj: ms_proj_t, bins: ms_bins_t, image_ptr: int,
             n_contrib_ptr: int, raster_ws_ptr: int, raster_ws_bytes: int,
             dl_ptr: int) -> ms_bwd_view_t:
    """One view of ms_raster_bwd_views (keeps no reference to proj/bins:
    the caller keeps them alive)."""
    return ms_bwd_view_t(cam, ctypes.pointer(proj), ctypes.pointer(bins), P(image_ptr),
                         P(n_contrib_ptr), P(raster_ws_ptr), raster_ws_bytes, P(dl_ptr))


def ms_raster_bwd_views(scene: ms_scene_t, views, grads: ms_grads_t, flags: int, ws_ptr: int,
                        ws_bytes: int, stream=None):
    arr = (ms_bwd_view_t * len(views))(*views)
    _check(lib().ms_raster_bwd_views(ctypes.byref(scene), arr, len(views), ctypes.byref(grads),
                                     int(flags), P(ws_ptr), ws_bytes, P(_stream(stream))))


def ms_l1_loss_grad(image_ptr: int, target_ptr: int, count: int, weight: float, dl_ptr: int,
                    loss_sum_ptr: int, stream=None):
    _check(lib().ms_l1_loss_grad(P(image_ptr), P(target_ptr), int(count), float(weight),
                                 P(dl_ptr), P(loss_sum_ptr), P(_stream(stream))))


def ms_aggregate_workspace_bytes(n: int) -> int:
    return int(lib().ms_aggregate_workspace_bytes(n))


def ms_aggregate(scene: ms_scene_t, cams, level_m: int, extent: float, out: ms_scene_t,
                 capacity: int, n_out_ptr: int, ws_ptr: int, ws_bytes: int, stream=None):
    arr = (ms_camera_t * max(len(cams), 1))(*cams)
    _check(lib().ms_aggregate(ctypes.byref(scene), arr, len(cams), int(level_m), float(extent),
                              ctypes.byref(out), int(capacity), P(n_out_ptr), P(ws_ptr),
                              ws_bytes, P(_stream(stream))))


def ms_serve_clock() -> float:
    return float(lib().ms_serve_clock())


def ms_serve_create(cfg: ms_serve_cfg_t) -> int:
    h = P()
    _check(lib().ms_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def ms_serve_add_scene(srv: int, scene: ms_scene_t) -> int:
    sid = ctypes.c_int32()
    _check(lib().ms_serve_add_scene(P(srv), ctypes.byref(scene), ctypes.byref(sid)))
    return sid.value


def ms_serve_submit(srv: int, req: ms_request_t) -> int:
    t = ctypes.c_uint64()
    _check(lib().ms_serve_submit(P(srv), ctypes.byref(req), ctypes.byref(t)))
    return t.value


def ms_serve_poll(srv: int, ticket: int) -> ms_result_t:
    r = ms_result_t()
    _check(lib().ms_serve_poll(P(srv), ticket, ctypes.byref(r)))
    return r


def ms_serve_wait(srv: int, ticket: int, timeout_s: float) -> ms_result_t:
    r = ms_result_t()
    _check(lib().ms_serve_wait(P(srv), ticket, float(timeout_s), ctypes.byref(r)))
    return r


def ms_serve_stats(srv: int) -> ms_serve_stats_t:
    st = ms_serve_stats_t()
    _check(lib().ms_serve_stats(P(srv), ctypes.byref(st)))
    return st


def ms_serve_destroy(srv: int):
    _check(lib().ms_serve_destroy(P(srv)))


# ------------------------------------------------------ buffer helpers

class DeviceScene:
    """A scene's arrays resident in device memory plus its ms_scene_t."""

    def __init__(self, scene: inputs.Scene, device="cuda", prepare: bool = True):
        import torch
        dev = torch.device(device)

        def f32(a):
            return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)

        self.n = scene.n
        self.n_levels = scene.n_levels
        self.sh_degree = scene.sh_degree
        self.mean = f32(scene.mean)
        self.log_scale = f32(scene.log_scale)
        self.quat = f32(scene.quat)
        self.opacity = f32(scene.opacity)
        self.color = f32(scene.color)
        self.level = torch.from_numpy(np.ascontiguousarray(scene.level, np.uint8)).to(dev)
        self.s_max = f32(scene.s_max)
        self.s_min = f32(scene.s_min)
        self.scale = torch.empty((max(self.n, 1), 3), dtype=torch.float32, device=dev)
        self.lnop = torch.empty(max(self.n, 1), dtype=torch.float32, device=dev)
        self.struct = ms_scene_t(
            self.n, self.n_levels, self.sh_degree, _ptr(self.mean), _ptr(self.log_scale),
            _ptr(self.quat), _ptr(self.opacity), _ptr(self.color), _ptr(self.level),
            _ptr(self.s_max), _ptr(self.s_min), _ptr(self.scale), _ptr(self.lnop))
        if prepare:
            ms_scene_prepare(self.struct)

    def set_range(self, s_max, s_min):
        import torch
        self.s_max.copy_(torch.as_tensor(np.ascontiguousarray(s_max, np.float32)))
        self.s_min.copy_(torch.as_tensor(np.ascontiguousarray(s_min, np.float32)))

    def calibrate(self, cams):
        """UpdateRange at each level's creation scale 4^(l-1) (Sec. 4.1) for
        every camera in order, on the device."""
        for cam in cams:
            for l in range(1, self.n_levels + 1):
                ms_update_range(self.struct, camera_struct(inputs.downscale(cam, 4 ** (l - 1))), l)


class Renderer:
    """Buffers for rendering one scene at images up to `max_tiles` tiles."""

    def __init__(self, n: int, max_tiles: int, dup_capacity: int, device="cuda",
                 with_cover: bool = True, with_mask: bool = True):
        import torch
        dev = torch.device(device)
        nn = max(n, 1)
        self.n = n
        self.max_tiles = max_tiles
        self.dup_capacity = dup_capacity
        self.rec = torch.empty(nn * REC_FLOATS, dtype=torch.float32, device=dev)
        self.rect = torch.empty(nn * 2, dtype=torch.int32, device=dev)
        self.n_tiles = torch.empty(nn, dtype=torch.int32, device=dev)
        self.depth = torch.empty(nn, dtype=torch.int32, device=dev)
        self.cover = torch.empty(nn, dtype=torch.float32, device=dev) if with_cover else None
        self.mask = (torch.empty((nn + 31) // 32, dtype=torch.int32, device=dev)
                     if with_mask else None)
        self.stats = torch.empty(MS_STATS_WORDS, dtype=torch.int32, device=dev)
        self.proj = ms_proj_t(_ptr(self.rec), _ptr(self.rect), _ptr(self.n_tiles),
                              _ptr(self.depth), _ptr(self.cover), _ptr(self.mask),
                              _ptr(self.stats), nn)
        self.gauss_idx = torch.empty(dup_capacity, dtype=torch.int32, device=dev)
        self.ranges = torch.empty(max_tiles * 2, dtype=torch.int32, device=dev)
        self.counts = torch.zeros(4, dtype=torch.int64, device=dev)
        self.bins = ms_bins_t(_ptr(self.gauss_idx), _ptr(self.ranges), _ptr(self.counts),
                              dup_capacity)
        self.ws_bytes = ms_bin_workspace_bytes(n, max_tiles, dup_capacity)
        if self.ws_bytes == 0:
            raise MsError(MS_ERR_INVALID_ARG, "invalid workspace sizes")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.rws_bytes = ms_raster_workspace_bytes(max_tiles, dup_capacity)
        if self.rws_bytes == 0:
            raise MsError(MS_ERR_INVALID_ARG, "invalid raster workspace sizes")
        self.rws = torch.empty(self.rws_bytes, dtype=torch.uint8, device=dev)

    def images(self, cam: inputs.Camera, device="cuda"):
        import torch
        H, W = cam.height, cam.width
        return (torch.empty((3, H, W), dtype=torch.float32, device=device),
                torch.empty((H, W), dtype=torch.float32, device=device),
                torch.empty((H, W), dtype=torch.int32, device=device))

    def render(self, scene: DeviceScene, cam: inputs.Camera, mode="selective", out=None,
               stream=None, n_eval=None, strategy="auto", max_ctas_per_sm=0):
        """Enqueue project -> bin -> raster.  Returns (image, final_t,
        n_contrib) device tensors; call `check()` after to learn D and
        whether the capacity sufficed.  `strategy` picks the raster kernel
        ("auto", "tile", "list", "group8/16/32", see ms_raster_ex) and
        max_ctas_per_sm caps the tile kernel's CTAs (ms_raster_ex2)."""
        if cam.tiles_x * cam.tiles_y > self.max_tiles:
            raise MsError(MS_ERR_INVALID_ARG, "camera has more tiles than max_tiles")
        ms_project(scene.struct, camera_struct(cam), MODES.get(mode, mode), self.proj, stream)
        return self.bin_raster(scene, cam, out, stream, n_eval, strategy,
                               max_ctas_per_sm=max_ctas_per_sm)

    def bin(self, scene: DeviceScene, cam: inputs.Camera, stream=None, order=None):
        """Enqueue the binning of this renderer's projection (left by
        ms_project or ms_project_views for `cam`).  With `order` (a
        DepthOrder sorted for a pose this frame shares, or (DepthOrder, v)
        for frame v of a split order) it takes that depth order instead of
        sorting (ms_bin_ordered)."""
        if cam.tiles_x * cam.tiles_y > self.max_tiles:
            raise MsError(MS_ERR_INVALID_ARG, "camera has more tiles than max_tiles")
        cs = camera_struct(cam)
        if order is None:
            ms_bin(self.proj, scene.n, cs, self.bins, _ptr(self.ws), self.ws_bytes, stream)
        else:
            order, v = order if isinstance(order, tuple) else (order, 0)
            o, st = order.view_order(v)
            ms_bin_ordered(self.proj, scene.n, cs, self.bins, o, st, _ptr(self.ws),
                           self.ws_bytes, stream)

    def raster(self, cam: inputs.Camera, out=None, stream=None, n_eval=None, strategy="auto",
               max_ctas_per_sm=0):
        """Enqueue the blend of this renderer's bins (ms_raster_ex2).
        Returns the (image, final_t, n_contrib) device tensors."""
        cs = camera_struct(cam)
        image, final_t, n_contrib = out if out is not None else self.images(cam)
        ms_raster_ex2(self.proj, self.bins, cs, _ptr(image), _ptr(final_t), _ptr(n_contrib),
                      _ptr(n_eval), _ptr(self.rws), self.rws_bytes,
                      STRATEGIES.get(strategy, strategy), max_ctas_per_sm, stream)
        return image, final_t, n_contrib

    def bin_raster(self, scene: DeviceScene, cam: inputs.Camera, out=None, stream=None,
                   n_eval=None, strategy="auto", order=None, max_ctas_per_sm=0):
        """Enqueue bin -> raster of this renderer's projection (see bin()
        and raster())."""
        self.bin(scene, cam, stream, order)
        return self.raster(cam, out, stream, n_eval, strategy, max_ctas_per_sm)

    def check(self, stream=None):
        rc, d, s = ms_bin_counts(self.bins, stream)
        if rc == MS_ERR_CAPACITY:
            raise MsError(rc, f"tile duplicates {d} exceed capacity {self.dup_capacity}")
        return d, s


class DepthOrder:
    """A depth order shared by the frames of one pose: the union of the
    Gaussians they list (ms_project_views_union), sorted once
    (ms_sort_depth) and consumed by each frame's ms_bin_ordered."""

    def __init__(self, n: int, device="cuda", split_views: int = 0):
        import torch
        dev = torch.device(device)
        nn = max(n, 1)
        self.n = n
        self.flags = torch.empty(nn, dtype=torch.int32, device=dev)
        self.stats = torch.empty(MS_STATS_WORDS, dtype=torch.int32, device=dev)
        self.order = torch.empty(nn, dtype=torch.int32, device=dev)
        self.ws_bytes = ms_sort_depth_workspace_bytes(n)
        if self.ws_bytes == 0:
            raise MsError(MS_ERR_INVALID_ARG, "invalid sort workspace size")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        # with split_views > 0: each view's own part of the order (ms_split_order)
        self.split_views = split_views
        self.view_orders = [torch.empty(nn, dtype=torch.int32, device=dev)
                            for _ in range(split_views)]
        self.view_stats = [torch.empty(MS_STATS_WORDS, dtype=torch.int32, device=dev)
                           for _ in range(split_views)]
        self.split_ws_bytes = ms_split_order_workspace_bytes(n) if split_views else 0
        self.split_ws = (torch.empty(max(self.split_ws_bytes, 16), dtype=torch.uint8, device=dev)
                         if split_views else None)

    def project(self, scene: "DeviceScene", renderers, cams, mode="selective", stream=None,
                views=None):
        """ms_project_views_union of cams (at most MS_MAX_PROJ_VIEWS) into
        renderers[v].proj, the union over `views` (indices of cameras of one
        pose; default all).  sort() then orders the union."""
        views = sorted(set(range(len(cams)) if views is None else views))
        if not views or views[0] < 0 or views[-1] >= len(cams):
            raise MsError(MS_ERR_INVALID_ARG, "views must index the cameras")
        ms_project_views_union(scene.struct, [camera_struct(c) for c in cams],
                               MODES.get(mode, mode), [r.proj for r in renderers],
                               sum(1 << v for v in views), _ptr(self.flags), _ptr(self.stats),
                               stream)
        u = renderers[views[0]].proj
        self._union = ms_proj_t(0, 0, _ptr(self.flags), u.depth, 0, 0, _ptr(self.stats), u.n)
        self._n = scene.n

    def sort(self, stream=None):
        """ms_sort_depth of the union formed by the last project(), then
        (split_views > 0) every view's own part of the order."""
        ms_sort_depth(self._union, self._n, _ptr(self.order), _ptr(self.ws), self.ws_bytes,
                      stream)
        if self.split_views:
            k = self.split_views
            ms_split_order(self._union, self._n, _ptr(self.order),
                           [_ptr(o) for o in self.view_orders[:k]],
                           [_ptr(t) for t in self.view_stats[:k]], _ptr(self.split_ws),
                           self.split_ws_bytes, stream)

    def view_order(self, v: int):
        """(order, order_stats) device pointers frame v bins from."""
        if self.split_views:
            return _ptr(self.view_orders[v]), _ptr(self.view_stats[v])
        return _ptr(self.order), _ptr(self.stats)


def depth_order_plan(survivors, frac: float = 0.8):
    """How the frames of one pose (survivors: their listed counts from an
    earlier pass) share one depth sort: (views, split).  When every frame
    lists at least `frac` of what the busiest lists, they all bin straight
    from the sorted union (split False: each skips the few Gaussians it
    does not list); otherwise the sorted union is split into every frame's
    own order (split True) rather than making the small frames skip through
    it."""
    views = list(range(len(survivors)))
    top = max(survivors) if len(survivors) else 0
    dense = top > 0 and min(survivors) >= frac * top
    return views, not dense


def shared_order_views(survivors, frac: float = 0.8):
    """The frames of a sweep worth binning from one shared depth order: those
    that list at least `frac` of the most any frame lists (their lists then
    overlap mostly, and each skips little of the union).  `survivors` are
    the frames' listed counts from an earlier pass."""
    top = max(survivors) if len(survivors) else 0
    return [v for v, s in enumerate(survivors) if top > 0 and s >= frac * top]


def share_ctas_per_sm(tiles: int, tiles_max: int) -> int:
    """CTAs per SM of the tile kernel for a frame of `tiles` tiles blended
    beside others (render_views with share_sms), the finest of them having
    tiles_max: 3 for the finest, one fewer for every 4x fewer tiles, at
    least 1, so that the blends leave the SMs room for the other frames'
    kernels in proportion to their work (on the 1M sweep the 1x, 2x and 4x
    frames at 3, 2, 1: 1.000-1.008 ms; at 2, 2, 2: 1.040-1.052 ms; at
    2, 2, 1: 1.009-1.020 ms; every CTA: 1.082-1.088 ms)."""
    import math
    steps = round(math.log(max(tiles_max, 1) / max(tiles, 1), 4)) if tiles > 0 else 3
    return max(1, 3 - steps)


def render_views(scene: DeviceScene, renderers, cams, mode="selective", outs=None,
                 streams=None, strategy="auto", order=None, order_views=None,
                 share_sms=False):
    """Several frames of one scene: one ms_project_views pass for every
    (up to MS_MAX_PROJ_VIEWS) cameras on the current stream, then each
    frame's bin -> raster on its own stream (streams[v], or the current
    stream), which the current stream waits for.  renderers[v] holds frame
    v's buffers.  With `order` (a DepthOrder; at most MS_MAX_PROJ_VIEWS
    cameras) the frames in order_views (default all; cameras of one pose)
    bin from one shared depth sort, the others sort their own lists.
    With share_sms (and streams), the frames the tile kernel blends (at
    least as many tiles as SMs) blend on share_ctas_per_sm() CTAs per SM,
    and the other frames start once those have binned, so that their
    binning and blending fill the SM room the fine frames' blends leave.
    Returns the (image, final_t, n_contrib) of every frame."""
    import torch
    n = len(cams)
    if (len(renderers) != n or (outs is not None and len(outs) != n)
            or (streams is not None and len(streams) != n)):
        raise MsError(MS_ERR_INVALID_ARG, "one renderer (and output and stream) per camera")
    for r, cam in zip(renderers, cams):
        if cam.tiles_x * cam.tiles_y > r.max_tiles:
            raise MsError(MS_ERR_INVALID_ARG, "camera has more tiles than max_tiles")
    main = torch.cuda.current_stream()
    m = MODES.get(mode, mode)
    if order is not None:
        if n > MS_MAX_PROJ_VIEWS:
            raise MsError(MS_ERR_INVALID_ARG, "a shared depth order covers at most "
                          f"{MS_MAX_PROJ_VIEWS} cameras")
        order_views = set(range(n) if order_views is None else order_views)
        order.project(scene, renderers, cams, m, main, order_views)
        sorted_ev = None
    else:
        for v0 in range(0, n, MS_MAX_PROJ_VIEWS):
            sl = slice(v0, min(n, v0 + MS_MAX_PROJ_VIEWS))
            ms_project_views(scene.struct, [camera_struct(c) for c in cams[sl]], m,
                             [r.proj for r in renderers[sl]], main)
    share = share_sms and streams is not None and strategy == "auto"
    sms = torch.cuda.get_device_properties(main.device).multi_processor_count if share else 0
    fine = [share and c.tiles_x * c.tiles_y >= sms for c in cams]
    tiles_max = max([c.tiles_x * c.tiles_y for c, f in zip(cams, fine) if f] or [1])
    binned = []   # events: the fine frames' binning done
    res = [None] * n
    for v in sorted(range(n), key=lambda k: not fine[k]):   # fine frames first
        r, cam = renderers[v], cams[v]
        st = streams[v] if streams is not None else main
        if st is not main:
            st.wait_stream(main)
        if order is not None and v in order_views:
            # the union is sorted on the stream of its first frame; the
            # union's other frames wait for the sort, the rest do not
            if sorted_ev is None:
                order.sort(st)
                sorted_ev = torch.cuda.Event()
                sorted_ev.record(st)
            else:
                st.wait_event(sorted_ev)
        if share and not fine[v]:
            for e in binned:
                st.wait_event(e)
        with torch.cuda.stream(st):
            r.bin(scene, cam, st, (order, v) if order is not None and v in order_views
                  else None)
            if fine[v]:
                binned.append(torch.cuda.Event())
                binned[-1].record(st)
            res[v] = r.raster(cam, None if outs is None else outs[v], st, strategy=strategy,
                              max_ctas_per_sm=(share_ctas_per_sm(cam.tiles_x * cam.tiles_y,
                                                                 tiles_max)
                                               if fine[v] else 0))
    if streams is not None:
        for st in streams:
            if st is not main:
                main.wait_stream(st)
    return res


def render(scene: inputs.Scene, cam: inputs.Camera, mode="selective", dup_capacity=None):
    """One-shot convenience: upload, render, return numpy (image, final_t,
    n_contrib).  Retries once with the exact duplicate count if the first
    capacity guess was too small."""
    import torch
    ds = DeviceScene(scene)
    cap = dup_capacity or max(1024, 8 * scene.n)
    for _ in range(2):
        r = Renderer(scene.n, cam.tiles_x * cam.tiles_y, cap)
        img, ft, nc = r.render(ds, cam, mode)
        rc, d, _ = ms_bin_counts(r.bins)
        if rc == MS_OK:
            torch.cuda.synchronize()
            return img.cpu().numpy(), ft.cpu().numpy(), nc.cpu().numpy()
        cap = d
    raise MsError(MS_ERR_CAPACITY, "duplicate capacity retry failed")


class Server:
    """A render server (ms_serve_*): resident DeviceScenes, requests
    submitted from any thread, results polled or awaited by ticket."""

    def __init__(self, max_gaussians: int, max_width: int, max_height: int,
                 mem_budget_bytes: int, max_inflight: int = 64, n_streams: int = 16,
                 initial_capacity: int = 0, device: int = 0, max_batch_views: int = 0):
        cfg = ms_serve_cfg_t(max_gaussians, max_width, max_height, max_inflight, n_streams,
                             mem_budget_bytes, initial_capacity, device, max_batch_views)
        self.handle = ms_serve_create(cfg)
        self.scenes = []   # keeps the DeviceScenes (their arrays) alive

    def add_scene(self, scene: "DeviceScene") -> int:
        sid = ms_serve_add_scene(self.handle, scene.struct)
        self.scenes.append(scene)
        return sid

    def submit(self, scene_id: int, cam: inputs.Camera, mode="selective", image_dev=None,
               image_host=None) -> int:
        req = ms_request_t(scene_id, MODES.get(mode, mode), camera_struct(cam),
                           _ptr(image_dev), _ptr(image_host))
        return ms_serve_submit(self.handle, req)

    def poll(self, ticket: int) -> ms_result_t:
        return ms_serve_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> ms_result_t:
        return ms_serve_wait(self.handle, ticket, timeout_s)

    def stats(self) -> ms_serve_stats_t:
        return ms_serve_stats(self.handle)

    def close(self):
        if self.handle:
            ms_serve_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def aggregate_level(scene: "DeviceScene", cams, level_m: int, extent: float,
                    capacity: int | None = None):
    """ms_aggregate for one coarse level: `cams` are inputs.Camera objects
    already downsampled by 4^(level_m - 1).  Returns the new Gaussians as a
    dict of device tensors (mean, log_scale, quat, opacity, color, level,
    s_max, s_min), in voxel-key order.  Synchronises (reads the count)."""
    import torch
    dev = scene.mean.device
    cap = max(1, scene.n if capacity is None else capacity)
    ws_bytes = ms_aggregate_workspace_bytes(scene.n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    n_out = torch.zeros(2, dtype=torch.int64, device=dev)
    for _ in range(2):
        o = dict(mean=torch.empty((cap, 3), device=dev), log_scale=torch.empty((cap, 3), device=dev),
                 quat=torch.empty((cap, 4), device=dev), opacity=torch.empty(cap, device=dev),
                 color=torch.empty((cap,) + tuple(scene.color.shape[1:]), device=dev),
                 level=torch.empty(cap, dtype=torch.uint8, device=dev),
                 s_max=torch.empty(cap, device=dev), s_min=torch.empty(cap, device=dev))
        out = ms_scene_t(cap, scene.n_levels, scene.sh_degree, _ptr(o["mean"]),
                         _ptr(o["log_scale"]), _ptr(o["quat"]), _ptr(o["opacity"]),
                         _ptr(o["color"]), _ptr(o["level"]), _ptr(o["s_max"]), _ptr(o["s_min"]),
                         0, 0)
        ms_aggregate(scene.struct, [camera_struct(c) for c in cams], level_m, extent, out, cap,
                     _ptr(n_out), _ptr(ws), ws_bytes)
        m, status = (int(v) for v in n_out.cpu())
        if status:
            raise MsError(MS_ERR_TIMEOUT, f"aggregate sort status {status:#x}")
        if m <= cap:
            return {k: v[:m] for k, v in o.items()}
        cap = m
    raise MsError(MS_ERR_CAPACITY, "aggregate capacity retry failed")
