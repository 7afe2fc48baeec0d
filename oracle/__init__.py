"""FP64/FP32 CPU oracle for multi-scale selective Gaussian splatting.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package.  It shares no code with the CUDA
library (paper_2311_17089_gb300); the two meet only through the seeded
inputs of paper_2311_17089_gb300.inputs.

The C sources (footprint32.c, render64.c, sh64.c, range.c, grad64.c) hold
the arithmetic; this module compiles them with gcc and marshals numpy
arrays through ctypes.

Parity unpinned: the paper's PSNR/LPIPS tables (datasets, trained models).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["footprint32.c", "render64.c", "sh64.c", "range.c", "grad64.c", "aggregate.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

SELECTIVE, ALL_LEVELS, FILTER_SMALL = 0, 1, 2
MODES = {"selective": SELECTIVE, "all_levels": ALL_LEVELS,
         "filter_small": FILTER_SMALL}

# Smallest relative margins around the blend's two thresholds inside which
# a single-precision evaluation may decide differently (flags, render64.c);
# each decision's margin is the larger of this floor and the bound of the
# single-precision error of the quantities it compares.
ALPHA_FLAG_REL = 1e-5
T_FLAG_REL = 1e-5
MAX_ALTERNATIVES = 256

FP_DTYPE = np.dtype([
    ("valid", np.uint8), ("selected", np.uint8), ("cover", np.float32),
    ("depth", np.uint32), ("rect", np.int32, (4,)), ("ntiles", np.uint32),
    ("ux", np.float32), ("uy", np.float32), ("conic", np.float32, (3,)),
], align=True)


class _Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("campos", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_plane", ctypes.c_float),
                ("bg", ctypes.c_float * 3)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FP contraction, no fast-math)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    newest = max(os.path.getmtime(p) for p in srcs + [os.path.join(_HERE, "oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I64, I32, D = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        L.or_prepare.argtypes = [I64, P, P, P, P]
        L.or_footprints32.argtypes = [I64, P, P, P, P, P, P, P, I32, I32, P, P]
        L.or_tile_lists.argtypes = [I64, P, I32, I32, P, P, I64]
        L.or_tile_lists.restype = I64
        L.or_sh_basis64.argtypes = [I32, P, P]
        L.or_colors64.argtypes = [I64, P, P, I32, P, P]
        L.or_render64.argtypes = [I64, P, P, P, P, P, P, P, I32, D, D, P, P, P, P, P]
        L.or_render64.restype = I64
        L.or_render64_brute.argtypes = [I64, P, P, P, P, D, P, P, P]
        L.or_render64_brute.restype = I64
        L.or_pixel_alternatives.argtypes = [P, P, P, P, I64, D, D, D, D, I32, P]
        L.or_pixel_alternatives.restype = I32
        L.or_update_range.argtypes = [I64, P, P, P, P, P, I32, I32, P, P, P]
        L.or_coverage64.argtypes = [I64, P, P, P, P, P, P, P, P, P]
        L.or_forward64_full.argtypes = [I64, P, P, P, P, P, I32, P, P, P, P, P, P, P]
        L.or_grad64.argtypes = [I64, P, P, P, P, P, I32, P, P, P, P, P, P, P, P, P]
        L.or_grad64.restype = I64
        L.or_voxel_key.argtypes = [P, ctypes.c_float, I32]
        L.or_voxel_key.restype = ctypes.c_uint32
        L.or_aggregate.argtypes = [I64, P, P, P, P, P, I32, P, P, P, I32, P, I32, ctypes.c_float,
                                   P, P, P, P, P, P, P, I64]
        L.or_aggregate.restype = I64
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "arrays passed to the oracle must be C-contiguous"
    return ctypes.c_void_p(a.ctypes.data)


def camera_struct(cam) -> _Camera:
    c = _Camera()
    c.R[:] = [float(v) for v in np.asarray(cam.R, np.float32).reshape(9)]
    c.t[:] = [float(v) for v in np.asarray(cam.t, np.float32)]
    c.campos[:] = [float(v) for v in np.asarray(cam.campos, np.float32)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = cam.width, cam.height
    c.near_plane = cam.near
    c.bg[:] = [float(v) for v in np.asarray(cam.bg, np.float32)]
    return c


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def prepare(scene):
    """exp(log_scale) and ln(255 sigma), FP64 rounded to FP32."""
    n = scene.n
    scale = np.empty((n, 3), np.float32)
    lnop = np.empty(n, np.float32)
    lib().or_prepare(n, _p(_f32(scene.log_scale)), _p(_f32(scene.opacity)),
                     _p(scale), _p(lnop))
    return scale, lnop


def footprints(scene, cam, mode="selective", prepared=None):
    scale, lnop = prepared if prepared is not None else prepare(scene)
    out = np.zeros(scene.n, FP_DTYPE)
    cs = camera_struct(cam)
    lib().or_footprints32(scene.n, _p(_f32(scene.mean)), _p(scale),
                          _p(_f32(scene.quat)), _p(lnop),
                          _p(np.ascontiguousarray(scene.level, np.uint8)),
                          _p(_f32(scene.s_max)), _p(_f32(scene.s_min)),
                          scene.n_levels, MODES.get(mode, mode),
                          ctypes.byref(cs), _p(out))
    return out


def tile_lists(fp, cam):
    tiles = cam.tiles_x * cam.tiles_y
    offsets = np.zeros(tiles + 1, np.int64)
    cap = int(np.sum(fp["ntiles"][fp["selected"] == 1], dtype=np.int64))
    idx = np.zeros(max(cap, 1), np.uint32)
    d = lib().or_tile_lists(len(fp), _p(fp), cam.tiles_x, cam.tiles_y,
                            _p(offsets), _p(idx), cap)
    assert d == cap
    return offsets, idx[:d]


def colors(scene, cam):
    rgb = np.empty((scene.n, 3), np.float64)
    cs = camera_struct(cam)
    lib().or_colors64(scene.n, _p(_f32(scene.mean)), _p(_f32(scene.color)),
                      scene.sh_degree, ctypes.byref(cs), _p(rgb))
    return rgb


def sh_basis(deg: int, direction) -> np.ndarray:
    d = np.ascontiguousarray(direction, np.float64)
    out = np.zeros((deg + 1) ** 2, np.float64)
    lib().or_sh_basis64(deg, _p(d), _p(out))
    return out


def render(scene, cam, mode="selective", tiles=None, prepared=None,
           alpha_flag_rel=ALPHA_FLAG_REL, t_flag_rel=T_FLAG_REL):
    """Full oracle render; `tiles` restricts it to a list of tile ids
    (the other pixels are left at NaN)."""
    fp = footprints(scene, cam, mode, prepared)
    offsets, idx = tile_lists(fp, cam)
    rgb = colors(scene, cam)
    H, W = cam.height, cam.width
    image = np.full((3, H, W), np.nan)
    final_t = np.full((H, W), np.nan)
    n_contrib = np.zeros((H, W), np.uint32)
    n_eval = np.zeros((H, W), np.int64)
    flags = np.zeros((H, W), np.uint8)
    cs = camera_struct(cam)
    sel = None
    if tiles is not None:
        sel = np.ascontiguousarray(tiles, np.int32)
    evals = lib().or_render64(
        scene.n, _p(fp), _p(_f32(scene.opacity)), _p(rgb), ctypes.byref(cs),
        _p(offsets), _p(idx if len(idx) else np.zeros(1, np.uint32)),
        _p(sel) if sel is not None else None,
        0 if sel is None else len(sel), alpha_flag_rel, t_flag_rel,
        _p(image), _p(final_t), _p(n_contrib), _p(flags), _p(n_eval))
    return dict(image=image, final_t=final_t, n_contrib=n_contrib,
                flags=flags, evals=int(evals), n_eval=n_eval, fp=fp, offsets=offsets,
                idx=idx, rgb=rgb, opacity=_f32(scene.opacity), cam=cam,
                alpha_flag_rel=alpha_flag_rel, t_flag_rel=t_flag_rel)


def pixel_alternatives(o, x: int, y: int, max_alts: int = MAX_ALTERNATIVES):
    """Every result pixel (x, y) of the render `o` (from render()) may take
    when its flagged decisions go either way: an array of rows (C0, C1, C2
    including T bg, T, n_contrib, n_eval), or None if there are more than
    max_alts.  The exact (FP64) decisions give one of the rows."""
    cam = o["cam"]
    t = (y // 16) * cam.tiles_x + x // 16
    off, idx = o["offsets"], o["idx"]
    lst = np.ascontiguousarray(idx[off[t]:off[t + 1]], np.uint32)
    out = np.zeros((max_alts, 6))
    k = lib().or_pixel_alternatives(
        _p(o["fp"]), _p(o["opacity"]), _p(o["rgb"]),
        _p(lst if len(lst) else np.zeros(1, np.uint32)), len(lst), x + 0.5, y + 0.5,
        o["alpha_flag_rel"], o["t_flag_rel"], max_alts, _p(out))
    if k < 0:
        return None
    out = out[:k]
    bg = np.asarray(cam.bg, np.float64)
    out[:, :3] += out[:, 3:4] * bg[None, :]
    return out


def render_brute(scene, cam, mode="selective", prepared=None,
                 alpha_flag_rel=ALPHA_FLAG_REL):
    fp = footprints(scene, cam, mode, prepared)
    rgb = colors(scene, cam)
    H, W = cam.height, cam.width
    image = np.zeros((3, H, W))
    final_t = np.zeros((H, W))
    flags = np.zeros((H, W), np.uint8)
    cs = camera_struct(cam)
    evals = lib().or_render64_brute(scene.n, _p(fp), _p(_f32(scene.opacity)),
                                    _p(rgb), ctypes.byref(cs), alpha_flag_rel,
                                    _p(image), _p(final_t), _p(flags))
    return dict(image=image, final_t=final_t, flags=flags, evals=int(evals),
                fp=fp)


def update_range(scene, cam, level_r: int, prepared=None):
    """Eq. 5 applied in place to scene.s_max / scene.s_min."""
    scale, lnop = prepared if prepared is not None else prepare(scene)
    cs = camera_struct(cam)
    smax = _f32(scene.s_max)
    smin = _f32(scene.s_min)
    lib().or_update_range(scene.n, _p(_f32(scene.mean)), _p(scale),
                          _p(_f32(scene.quat)), _p(lnop),
                          _p(np.ascontiguousarray(scene.level, np.uint8)),
                          scene.n_levels, level_r, ctypes.byref(cs),
                          _p(smax), _p(smin))
    scene.s_max, scene.s_min = smax, smin


def calibrate(scene, cams):
    """Coverage ranges as multi-scale training would leave them: for each
    camera in order, every level l is rendered at its creation scale
    4^(l-1) (Sec. 4.1) and UpdateRange (Eq. 5) applied to that level."""
    from paper_2311_17089_gb300.inputs import downscale
    prepared = prepare(scene)
    for cam in cams:
        for l in range(1, scene.n_levels + 1):
            update_range(scene, downscale(cam, 4 ** (l - 1)), l, prepared)
    return scene


def coverage64(scene, cam):
    n = scene.n
    cover = np.empty(n)
    ux = np.empty(n)
    uy = np.empty(n)
    cov2d = np.empty((n, 3))
    cs = camera_struct(cam)
    lib().or_coverage64(n, _p(_f32(scene.mean)), _p(_f32(scene.log_scale)),
                        _p(_f32(scene.quat)), _p(_f32(scene.opacity)),
                        ctypes.byref(cs), _p(cover), _p(ux), _p(uy), _p(cov2d))
    return cover, ux, uy, cov2d


def forward64(scene, cam, offsets, idx):
    """FP64 render with an FP64 projection over fixed tile lists (the
    function the gradient differentiates)."""
    H, W = cam.height, cam.width
    image = np.zeros((3, H, W))
    final_t = np.zeros((H, W))
    n_contrib = np.zeros((H, W), np.uint32)
    n_blend = np.zeros((H, W), np.uint32)
    cs = camera_struct(cam)
    lib().or_forward64_full(scene.n, _p(_f32(scene.mean)), _p(_f32(scene.log_scale)),
                            _p(_f32(scene.quat)), _p(_f32(scene.opacity)),
                            _p(_f32(scene.color)), scene.sh_degree, ctypes.byref(cs),
                            _p(np.ascontiguousarray(offsets, np.int64)),
                            _p(np.ascontiguousarray(idx if len(idx) else np.zeros(1), np.uint32)),
                            _p(image), _p(final_t), _p(n_contrib), _p(n_blend))
    return dict(image=image, final_t=final_t, n_contrib=n_contrib, n_blend=n_blend)


def grad64(scene, cam, offsets, idx, dl_dimage):
    """Analytic FP64 gradient of sum(dl_dimage * image) with respect to
    mean, log_scale, quat, opacity and colour (tile lists held fixed)."""
    n = scene.n
    g = dict(mean=np.zeros((n, 3)), log_scale=np.zeros((n, 3)), quat=np.zeros((n, 4)),
             opacity=np.zeros(n), color=np.zeros(scene.color.shape))
    cs = camera_struct(cam)
    lib().or_grad64(n, _p(_f32(scene.mean)), _p(_f32(scene.log_scale)), _p(_f32(scene.quat)),
                    _p(_f32(scene.opacity)), _p(_f32(scene.color)), scene.sh_degree,
                    ctypes.byref(cs), _p(np.ascontiguousarray(offsets, np.int64)),
                    _p(np.ascontiguousarray(idx if len(idx) else np.zeros(1), np.uint32)),
                    _p(np.ascontiguousarray(dl_dimage, np.float64)), _p(g["mean"]),
                    _p(g["log_scale"]), _p(g["quat"]), _p(g["opacity"]), _p(g["color"]))
    return g


def voxel_key(mean3, B: float, level_m: int) -> int:
    m = np.ascontiguousarray(mean3, np.float32)
    return int(lib().or_voxel_key(_p(m), float(B), int(level_m)))


def aggregate(scene, cams, level_m: int, B: float):
    """AggregateGaussians (Alg. 1) for level l_m: cams are the training
    cameras already downsampled by 4^(l_m-1).  Returns (new Gaussians as a
    dict of arrays in voxel-key order, their voxel keys, smallest coverage
    per input Gaussian)."""
    n = scene.n
    scale, lnop = prepare(scene)
    K = 1 if scene.sh_degree < 0 else (scene.sh_degree + 1) ** 2
    cam_arr = (_Camera * max(len(cams), 1))(*[camera_struct(c) for c in cams])
    smin = np.empty(max(n, 1), np.float32)
    cap = max(n, 1)
    out = dict(mean=np.zeros((cap, 3), np.float32), log_scale=np.zeros((cap, 3), np.float32),
               quat=np.zeros((cap, 4), np.float32), opacity=np.zeros(cap, np.float32),
               color=np.zeros((cap,) + scene.color.shape[1:], np.float32))
    keys = np.zeros(cap, np.uint32)
    m = lib().or_aggregate(n, _p(_f32(scene.mean)), _p(_f32(scene.log_scale)),
                           _p(_f32(scene.quat)), _p(_f32(scene.opacity)), _p(_f32(scene.color)),
                           scene.sh_degree, _p(np.ascontiguousarray(scene.level, np.uint8)),
                           _p(scale), _p(lnop), len(cams), cam_arr, level_m, float(B),
                           _p(smin), _p(out["mean"]), _p(out["log_scale"]), _p(out["quat"]),
                           _p(out["opacity"]), _p(out["color"]), _p(keys), cap)
    return {k: v[:m] for k, v in out.items()}, keys[:m], smin[:n]
