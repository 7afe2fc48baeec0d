"""torch.autograd glue for differentiable rendering through libmsgs.

Marshalling only: the forward is ms_scene_prepare -> ms_project -> ms_bin
-> ms_raster and the backward is ms_raster_bwd, all CUDA kernels of
libmsgs.so.  A `Frame` owns one frame's device buffers (projection, tile
lists, image, contributor counts, raster workspace), which the backward of
that frame needs, so every camera of a batch uses its own Frame.
"""
from __future__ import annotations

import torch

from . import (MODES, STRATEGIES, MsError, MS_OK, MS_MAX_BWD_VIEWS, Renderer, _ptr, bwd_view,
               camera_struct, ms_bin, ms_bin_counts, ms_grads_t, ms_project, ms_raster_ex2,
               ms_raster_bwd, ms_raster_bwd_views, ms_raster_bwd_views_workspace_bytes,
               ms_raster_bwd_workspace_bytes, ms_scene_prepare, ms_scene_t)
from . import inputs


class Frame:
    """Buffers for rendering and differentiating one view.  `strategy`
    picks the forward's raster kernel ("auto", "tile", "list", "group8/16/32",
    ms_raster_ex; "tile@K": the tile kernel on at most K CTAs per SM,
    ms_raster_ex2); the backward reads any one's segment states."""

    def __init__(self, n: int, cam: inputs.Camera, dup_capacity: int, device="cuda",
                 strategy="auto"):
        self.cam = cam
        name, _, ctas = strategy.partition("@") if isinstance(strategy, str) else (strategy, "", "")
        self.strategy = STRATEGIES.get(name, name)
        self.max_ctas_per_sm = int(ctas) if ctas else 0
        self.renderer = Renderer(n, cam.tiles_x * cam.tiles_y, dup_capacity, device=device,
                                 with_cover=False, with_mask=False)
        self.image, self.final_t, self.n_contrib = self.renderer.images(cam, device=device)
        self.bwd_ws_bytes = ms_raster_bwd_workspace_bytes(n)
        self.bwd_ws = torch.empty(self.bwd_ws_bytes, dtype=torch.uint8, device=device)


def _scene_struct(n, n_levels, sh_degree, mean, log_scale, quat, opacity, color, level, s_max,
                  s_min, scale, lnop):
    return ms_scene_t(n, n_levels, sh_degree, _ptr(mean), _ptr(log_scale), _ptr(quat),
                      _ptr(opacity), _ptr(color), _ptr(level), _ptr(s_max), _ptr(s_min),
                      _ptr(scale), _ptr(lnop))


class GaussianRender(torch.autograd.Function):
    """image = render(mean, log_scale, quat, opacity, color) for one camera.

    level, s_max, s_min select Gaussians (Eq. 6) and are not differentiated.
    """

    @staticmethod
    def forward(ctx, mean, log_scale, quat, opacity, color, level, s_max, s_min, n_levels,
                sh_degree, mode, frame: Frame):
        mean, log_scale, quat, opacity, color = (t.contiguous() for t in
                                                 (mean, log_scale, quat, opacity, color))
        n = mean.shape[0]
        scale = torch.empty_like(log_scale)
        lnop = torch.empty_like(opacity)
        sc = _scene_struct(n, n_levels, sh_degree, mean, log_scale, quat, opacity, color,
                           level, s_max, s_min, scale, lnop)
        ms_scene_prepare(sc)
        r = frame.renderer
        cs = camera_struct(frame.cam)
        ms_project(sc, cs, MODES.get(mode, mode), r.proj)
        ms_bin(r.proj, n, cs, r.bins, _ptr(r.ws), r.ws_bytes)
        ms_raster_ex2(r.proj, r.bins, cs, _ptr(frame.image), _ptr(frame.final_t),
                      _ptr(frame.n_contrib), 0, _ptr(r.rws), r.rws_bytes, frame.strategy,
                      frame.max_ctas_per_sm)
        ctx.frame = frame
        ctx.meta = (n, n_levels, sh_degree)
        ctx.save_for_backward(mean, log_scale, quat, opacity, color, level, s_max, s_min,
                              scale, lnop)
        return frame.image.clone()

    @staticmethod
    def backward(ctx, grad_image):
        (mean, log_scale, quat, opacity, color, level, s_max, s_min, scale,
         lnop) = ctx.saved_tensors
        n, n_levels, sh_degree = ctx.meta
        frame = ctx.frame
        r = frame.renderer
        g = {k: torch.empty_like(t) for k, t in (("mean", mean), ("log_scale", log_scale),
                                                 ("quat", quat), ("opacity", opacity),
                                                 ("color", color))}
        sc = _scene_struct(n, n_levels, sh_degree, mean, log_scale, quat, opacity, color,
                           level, s_max, s_min, scale, lnop)
        grads = ms_grads_t(_ptr(g["mean"]), _ptr(g["log_scale"]), _ptr(g["quat"]),
                           _ptr(g["opacity"]), _ptr(g["color"]))
        ms_raster_bwd(sc, camera_struct(frame.cam), r.proj, r.bins, _ptr(frame.image),
                      _ptr(frame.n_contrib), _ptr(r.rws), r.rws_bytes,
                      _ptr(grad_image.contiguous()), grads, 0, _ptr(frame.bwd_ws),
                      frame.bwd_ws_bytes)
        return (g["mean"], g["log_scale"], g["quat"], g["opacity"], g["color"], None, None,
                None, None, None, None, None)


class GaussianRenderViews(torch.autograd.Function):
    """(image_1, ..., image_k) = render(params) for k cameras (one Frame
    each) of the same scene; the backward of all views is one
    ms_raster_bwd_views call."""

    @staticmethod
    def forward(ctx, mean, log_scale, quat, opacity, color, level, s_max, s_min, n_levels,
                sh_degree, mode, frames):
        if not 1 <= len(frames) <= MS_MAX_BWD_VIEWS:
            raise ValueError(f"1..{MS_MAX_BWD_VIEWS} frames")
        mean, log_scale, quat, opacity, color = (t.contiguous() for t in
                                                 (mean, log_scale, quat, opacity, color))
        n = mean.shape[0]
        scale = torch.empty_like(log_scale)
        lnop = torch.empty_like(opacity)
        sc = _scene_struct(n, n_levels, sh_degree, mean, log_scale, quat, opacity, color,
                           level, s_max, s_min, scale, lnop)
        ms_scene_prepare(sc)
        outs = []
        for frame in frames:
            r = frame.renderer
            cs = camera_struct(frame.cam)
            ms_project(sc, cs, MODES.get(mode, mode), r.proj)
            ms_bin(r.proj, n, cs, r.bins, _ptr(r.ws), r.ws_bytes)
            ms_raster_ex2(r.proj, r.bins, cs, _ptr(frame.image), _ptr(frame.final_t),
                          _ptr(frame.n_contrib), 0, _ptr(r.rws), r.rws_bytes, frame.strategy,
                          frame.max_ctas_per_sm)
            outs.append(frame.image.clone())
        ctx.frames = frames
        ctx.meta = (n, n_levels, sh_degree)
        ctx.save_for_backward(mean, log_scale, quat, opacity, color, level, s_max, s_min,
                              scale, lnop)
        return tuple(outs)

    @staticmethod
    def backward(ctx, *grad_images):
        (mean, log_scale, quat, opacity, color, level, s_max, s_min, scale,
         lnop) = ctx.saved_tensors
        n, n_levels, sh_degree = ctx.meta
        g = {k: torch.empty_like(t) for k, t in (("mean", mean), ("log_scale", log_scale),
                                                 ("quat", quat), ("opacity", opacity),
                                                 ("color", color))}
        sc = _scene_struct(n, n_levels, sh_degree, mean, log_scale, quat, opacity, color,
                           level, s_max, s_min, scale, lnop)
        grads = ms_grads_t(_ptr(g["mean"]), _ptr(g["log_scale"]), _ptr(g["quat"]),
                           _ptr(g["opacity"]), _ptr(g["color"]))
        dls = [(gi if gi is not None else torch.zeros_like(f.image)).contiguous()
               for gi, f in zip(grad_images, ctx.frames)]
        views = [bwd_view(camera_struct(f.cam), f.renderer.proj, f.renderer.bins,
                          _ptr(f.image), _ptr(f.n_contrib), _ptr(f.renderer.rws),
                          f.renderer.rws_bytes, _ptr(dl)) for f, dl in zip(ctx.frames, dls)]
        wsb = ms_raster_bwd_views_workspace_bytes(n, len(views))
        ws = torch.empty(wsb, dtype=torch.uint8, device=mean.device)
        ms_raster_bwd_views(sc, views, grads, 0, _ptr(ws), wsb)
        return (g["mean"], g["log_scale"], g["quat"], g["opacity"], g["color"], None, None,
                None, None, None, None, None)


def render_views(params: dict, level, s_max, s_min, n_levels: int, sh_degree: int, frames,
                 mode="selective"):
    """Differentiable render of several views (one Frame each); returns a
    tuple of images whose backward is one batched call."""
    return GaussianRenderViews.apply(params["mean"], params["log_scale"], params["quat"],
                                     params["opacity"], params["color"], level, s_max, s_min,
                                     n_levels, sh_degree, mode, list(frames))


def render(params: dict, level, s_max, s_min, n_levels: int, sh_degree: int, frame: Frame,
           mode="selective"):
    """Differentiable render of one view; `params` holds the tensors mean,
    log_scale, quat, opacity and color (any may require grad)."""
    return GaussianRender.apply(params["mean"], params["log_scale"], params["quat"],
                                params["opacity"], params["color"], level, s_max, s_min,
                                n_levels, sh_degree, mode, frame)


def check_frame(frame: Frame):
    """Duplicate count of the frame's last forward; raises if the capacity
    was too small (synchronises)."""
    rc, d, _ = ms_bin_counts(frame.renderer.bins)
    if rc != MS_OK:
        raise MsError(rc, f"tile duplicates {d} exceed capacity {frame.renderer.dup_capacity}")
    return d
