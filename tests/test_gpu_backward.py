"""Parity of the CUDA backward (ms_raster_bwd, through the C ABI and the
autograd glue) with the oracle's FP64 analytic gradient and with central
finite differences of the oracle's FP64 forward."""
import numpy as np
import pytest

import oracle
from paper_2311_17089_gb300 import autograd as ag
from paper_2311_17089_gb300 import inputs

from gpu_util import require_cuda

pytestmark = pytest.mark.gpu
NAMES = ("mean", "log_scale", "quat", "opacity", "color")


def gpu_grads(sc, cam, w, mode="all_levels", strategy="auto"):
    torch = require_cuda()
    dev = torch.device("cuda")
    params = {k: torch.tensor(np.ascontiguousarray(getattr(sc, k), np.float32), device=dev,
                              requires_grad=True) for k in NAMES}
    level = torch.tensor(sc.level, device=dev)
    smax = torch.tensor(sc.s_max, device=dev)
    smin = torch.tensor(sc.s_min, device=dev)
    frame = ag.Frame(sc.n, cam, max(4096, 64 * sc.n), device=dev, strategy=strategy)
    img = ag.render(params, level, smax, smin, sc.n_levels, sc.sh_degree, frame, mode)
    ag.check_frame(frame)
    loss = (img * torch.tensor(w, dtype=torch.float32, device=dev)).sum()
    loss.backward()
    torch.cuda.synchronize()
    return {k: params[k].grad.detach().cpu().numpy().astype(np.float64) for k in NAMES}, img


GRAD_LOG = []   # (test case, parameter, entries, entries within rel only through the floor)


def compare(gg, go, rel=1e-3, floor=1e-4):
    """Each entry within rel of the oracle's value plus a floor relative to
    the largest entry of that parameter.  The floor covers entries that are
    small sums of larger terms (FP32 accumulation over many pixels cancels)
    and Gaussians that touch pixels whose threshold decisions the FP32 path
    and the FP64 oracle take differently; the entries that pass only
    through it are counted (GRAD_LOG, printed at the end of the run)."""
    import os
    case = os.environ.get("PYTEST_CURRENT_TEST", "grad").split(" ")[0]
    for k in NAMES:
        a, b = gg[k].reshape(-1), go[k].reshape(-1)
        scale = max(np.abs(b).max(), 1e-30)
        err = np.abs(a - b)
        bad = err > rel * np.abs(b) + floor * scale
        assert not bad.any(), (k, int(bad.sum()), float((err / scale).max()))
        GRAD_LOG.append((case, k, int(a.size), int((err > rel * np.abs(b)).sum())))


@pytest.mark.parametrize("strategy", ["tile", "tile@1", "list", "group8", "group16", "group32"])
@pytest.mark.parametrize("seed,deg,n,size", [(0, -1, 64, 64), (1, 3, 64, 64), (2, 1, 400, 96),
                                              (3, 3, 3000, 160)])
def test_backward_matches_oracle_gradient(seed, deg, n, size, strategy):
    """The backward after either raster kernel's forward."""
    sc = inputs.tiny_scene(n=n, seed=seed, sh_degree=deg, extent=0.8 if n > 100 else 0.6)
    cam = inputs.config1_camera(size, size)
    cam.bg[:] = [0.2, 0.3, 0.1]
    w = np.random.default_rng(seed).standard_normal((3, size, size))
    gg, _ = gpu_grads(sc, cam, w, strategy=strategy)
    fp = oracle.footprints(sc, cam, "all_levels")
    off, idx = oracle.tile_lists(fp, cam)
    go = oracle.grad64(sc, cam, off, idx, w)
    compare(gg, go)


@pytest.mark.parametrize("strategy", ["tile", "tile@1", "tile@2", "list", "group8", "group16",
                                      "group32"])
def test_backward_long_lists_many_segments(strategy):
    """Thousands of faint, wide Gaussians on a 48x32 frame (6 tiles): every
    tile's list spans several segments, so the backward starts most
    segments from the prefix state the forward stored at its start (the
    list kernel stores it at each segment boundary a pixel passes, the tile
    kernel when it publishes the segment).  Pixels terminate in later
    segments (opacity ~0.01)."""
    rng = np.random.default_rng(11)
    n = 4000
    mean = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.4, 0.4, n),
                     rng.uniform(-1.0, 1.0, n)], 1).astype(np.float32)
    log_scale = rng.normal(np.log(6.0), 0.05, (n, 3)).astype(np.float32)
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    opacity = rng.uniform(0.008, 0.014, n).astype(np.float32)
    color = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    sc = inputs.Scene(mean, log_scale, quat, opacity, color, np.ones(n, np.uint8), 1, -1,
                      np.zeros(n, np.float32), np.full(n, np.inf, np.float32))
    cam = inputs.config1_camera(48, 32)
    fp = oracle.footprints(sc, cam, "all_levels")
    off, idx = oracle.tile_lists(fp, cam)
    assert np.diff(off).min() > 4 * 256    # several 256-entry segments per tile
    w = rng.standard_normal((3, 32, 48))
    gg, _ = gpu_grads(sc, cam, w, strategy=strategy)
    go = oracle.grad64(sc, cam, off, idx, w)
    compare(gg, go)


@pytest.mark.parametrize("strategy", ["tile", "list", "group8", "group16", "group32"])
def test_backward_deep_lists(strategy):
    """The backward on 7.5k-8.3k-entry lists where half of the pixels
    terminate early and the other half blend far down the list."""
    from test_gpu_parity import deep_lists_scene
    sc = deep_lists_scene(seed=32)
    cam = inputs.config1_camera(48, 32)
    w = np.random.default_rng(33).standard_normal((3, 32, 48))
    gg, _ = gpu_grads(sc, cam, w, strategy=strategy)
    fp = oracle.footprints(sc, cam, "all_levels")
    off, idx = oracle.tile_lists(fp, cam)
    assert np.diff(off).min() > 4096
    go = oracle.grad64(sc, cam, off, idx, w)
    compare(gg, go)


def test_backward_lists_past_the_mask_prefix():
    """The backward after the list kernel on lists longer than its mask
    pass's 16384-entry prefix (the forward's prefix states past it come
    from entries whose masks the blend formed itself)."""
    from test_gpu_parity import deep_lists_scene
    sc = deep_lists_scene(seed=36, nb=110_000)
    cam = inputs.config1_camera(48, 32)
    w = np.random.default_rng(37).standard_normal((3, 32, 48))
    gg, _ = gpu_grads(sc, cam, w, strategy="list")
    fp = oracle.footprints(sc, cam, "all_levels")
    off, idx = oracle.tile_lists(fp, cam)
    assert np.diff(off).min() > 16384 + 1024
    go = oracle.grad64(sc, cam, off, idx, w)
    compare(gg, go)


def test_backward_multiscale_selective():
    sc = inputs.multiscale_scene(n=20_000, seed=2, box=2.0, cluster_sigma=0.5, n_clusters=16)
    cam = inputs.config2_camera(256, 192, distance=6.0)
    sc = oracle.calibrate(sc, inputs.orbit_cameras(4, seed=3, radius=6.0, width=256, height=192))
    w = np.random.default_rng(7).standard_normal((3, 192, 256))
    gg, _ = gpu_grads(sc, cam, w, "selective")
    fp = oracle.footprints(sc, cam, "selective")
    off, idx = oracle.tile_lists(fp, cam)
    go = oracle.grad64(sc, cam, off, idx, w)
    compare(gg, go)


def test_backward_matches_finite_differences():
    """Central differences of the FP64 forward against the CUDA gradient."""
    sc = inputs.tiny_scene(n=48, seed=4, sh_degree=3)
    cam = inputs.config1_camera(48, 48)
    rng = np.random.default_rng(4)
    w = rng.standard_normal((3, 48, 48))
    gg, _ = gpu_grads(sc, cam, w)
    fp = oracle.footprints(sc, cam, "all_levels")
    off, idx = oracle.tile_lists(fp, cam)
    base = oracle.forward64(sc, cam, off, idx)
    sig0 = (base["n_contrib"], base["n_blend"])
    checked = 0
    for k, h in (("mean", 1e-4), ("log_scale", 1e-4), ("quat", 1e-4), ("opacity", 1e-4),
                 ("color", 1e-3)):
        arr = getattr(sc, k).reshape(-1)
        g = gg[k].reshape(-1)
        scale = np.abs(g).max()
        cand = np.nonzero(np.abs(g) > 1e-3 * scale)[0]
        for j in rng.choice(cand, min(8, len(cand)), replace=False):
            th = arr[j]
            tp, tm = np.float32(th + h), np.float32(th - h)
            arr[j] = tp
            rp = oracle.forward64(sc, cam, off, idx)
            arr[j] = tm
            rm = oracle.forward64(sc, cam, off, idx)
            arr[j] = th
            if not (np.array_equal(rp["n_contrib"], sig0[0]) and np.array_equal(rm["n_contrib"], sig0[0])
                    and np.array_equal(rp["n_blend"], sig0[1]) and np.array_equal(rm["n_blend"], sig0[1])):
                continue
            fd = float(np.sum(w * rp["image"]) - np.sum(w * rm["image"])) / (float(tp) - float(tm))
            assert abs(fd - g[j]) <= 1e-3 * abs(fd) + 1e-4 * scale, (k, j, fd, g[j])
            checked += 1
    assert checked >= 30


def test_training_step_reduces_l1_loss():
    """A few Adam steps on an L1 loss against a target rendered from a
    perturbed scene reduce the loss (the gradient has the right sign end to
    end)."""
    torch = require_cuda()
    dev = torch.device("cuda")
    sc = inputs.tiny_scene(n=200, seed=6, sh_degree=1, extent=0.8)
    cam = inputs.config1_camera(96, 96)
    target_scene = sc.copy()
    target_scene.color = (target_scene.color * 0.5).astype(np.float32)
    frame_t = ag.Frame(sc.n, cam, 64 * sc.n, device=dev)
    tp = {k: torch.tensor(getattr(target_scene, k), device=dev) for k in NAMES}
    level = torch.tensor(sc.level, device=dev)
    smax = torch.tensor(sc.s_max, device=dev)
    smin = torch.tensor(sc.s_min, device=dev)
    target = ag.render(tp, level, smax, smin, 1, 1, frame_t, "all_levels").detach()
    params = {k: torch.tensor(getattr(sc, k), device=dev, requires_grad=True) for k in NAMES}
    opt = torch.optim.Adam([params["color"]], lr=0.02)
    frame = ag.Frame(sc.n, cam, 64 * sc.n, device=dev)
    losses = []
    for _ in range(20):
        opt.zero_grad()
        img = ag.render(params, level, smax, smin, 1, 1, frame, "all_levels")
        loss = (img - target).abs().mean()
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < 0.5 * losses[0], losses


def _bwd_raw(sc, cams, flags_seq, ws_list):
    """Forward each camera through the C ABI, then ms_raster_bwd with the
    given flags into ONE set of gradient buffers; returns host grads."""
    torch = require_cuda()
    import paper_2311_17089_gb300 as msgs
    ds = msgs.DeviceScene(sc)
    g = {k: torch.full(np.shape(getattr(sc, k)), 7.0, device="cuda") for k in NAMES}
    grads = msgs.ms_grads_t(*(msgs._ptr(g[k]) for k in NAMES))
    for cam, flags, w in zip(cams, flags_seq, ws_list):
        r = msgs.Renderer(sc.n, cam.tiles_x * cam.tiles_y, 64 * sc.n, with_cover=False,
                          with_mask=False)
        img, ft, nc = r.render(ds, cam, "all_levels")
        r.check()
        dl = torch.tensor(w, dtype=torch.float32, device="cuda")
        ws = torch.empty(msgs.ms_raster_bwd_workspace_bytes(sc.n), dtype=torch.uint8,
                         device="cuda")
        msgs.ms_raster_bwd(ds.struct, msgs.camera_struct(cam), r.proj, r.bins, msgs._ptr(img),
                           msgs._ptr(nc), msgs._ptr(r.rws), r.rws_bytes, msgs._ptr(dl), grads,
                           flags, msgs._ptr(ws), ws.numel())
        torch.cuda.synchronize()
    return {k: g[k].cpu().numpy().astype(np.float64) for k in NAMES}


def test_backward_accumulates_over_views():
    """flags = MS_BWD_ACCUMULATE adds a view's gradient: overwrite + add
    over two views equals the sum of the oracle's per-view gradients."""
    import paper_2311_17089_gb300 as msgs
    sc = inputs.tiny_scene(n=300, seed=9, sh_degree=2, extent=0.8)
    cams = [inputs.config1_camera(80, 64)] + inputs.orbit_cameras(1, seed=1, radius=3.0,
                                                                    width=48, height=48)
    rng = np.random.default_rng(9)
    ws = [rng.standard_normal((3, c.height, c.width)) for c in cams]
    gg = _bwd_raw(sc, cams, [0, msgs.MS_BWD_ACCUMULATE], ws)
    go = {k: 0.0 for k in NAMES}
    for cam, w in zip(cams, ws):
        fp = oracle.footprints(sc, cam, "all_levels")
        off, idx = oracle.tile_lists(fp, cam)
        g1 = oracle.grad64(sc, cam, off, idx, w)
        go = {k: go[k] + g1[k] for k in NAMES}
    compare(gg, go)
    # overwrite mode clears stale values (buffers start at 7.0)
    g0 = _bwd_raw(sc, cams[1:], [0], ws[1:])
    assert np.all(np.isfinite(g0["color"])) and np.abs(g0["color"]).max() < 7.0


def test_l1_loss_grad_kernel():
    torch = require_cuda()
    import paper_2311_17089_gb300 as msgs
    rng = np.random.default_rng(3)
    count = 3 * 37 * 41                       # not a multiple of 4: ragged tail
    a = rng.uniform(0, 1, count).astype(np.float32)
    b = rng.uniform(0, 1, count).astype(np.float32)
    b[::7] = a[::7]                           # exact ties: sign 0
    img, tgt = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    dl = torch.empty_like(img)
    loss = torch.zeros(1, device="cuda")
    wgt = np.float32(1.0 / count)
    msgs.ms_l1_loss_grad(msgs._ptr(img), msgs._ptr(tgt), count, float(wgt), msgs._ptr(dl),
                         msgs._ptr(loss))
    msgs.ms_l1_loss_grad(msgs._ptr(img), msgs._ptr(tgt), count, float(wgt), msgs._ptr(dl),
                         msgs._ptr(loss))
    torch.cuda.synchronize()
    d = a.astype(np.float64) - b
    assert np.array_equal(dl.cpu().numpy(), (np.sign(d) * wgt).astype(np.float32))
    assert float(loss) == pytest.approx(2 * float(wgt) * np.abs(d).sum(), rel=1e-5)


def test_batched_views_backward_matches_oracle_sum():
    """ms_raster_bwd_views over three views of different sizes (one
    launch per stage) equals the sum of the oracle's per-view gradients."""
    torch = require_cuda()
    import paper_2311_17089_gb300 as msgs
    sc = inputs.tiny_scene(n=500, seed=11, sh_degree=3, extent=0.8)
    cams = [inputs.config1_camera(96, 80)] + inputs.orbit_cameras(
        2, seed=4, radius=3.0, width=64, height=48)
    cams[2] = inputs.downscale(cams[2], 2)
    rng = np.random.default_rng(12)
    ws_ = [rng.standard_normal((3, c.height, c.width)) for c in cams]
    ds = msgs.DeviceScene(sc)
    keep, views = [], []
    for cam, w in zip(cams, ws_):
        r = msgs.Renderer(sc.n, cam.tiles_x * cam.tiles_y, 64 * sc.n, with_cover=False,
                          with_mask=False)
        img, ft, nc = r.render(ds, cam, "all_levels")
        r.check()
        dl = torch.tensor(w, dtype=torch.float32, device="cuda")
        keep.append((r, img, nc, dl))
        views.append(msgs.bwd_view(msgs.camera_struct(cam), r.proj, r.bins, msgs._ptr(img),
                                   msgs._ptr(nc), msgs._ptr(r.rws), r.rws_bytes, msgs._ptr(dl)))
    g = {k: torch.full(np.shape(getattr(sc, k)), 3.0, device="cuda") for k in NAMES}
    grads = msgs.ms_grads_t(*(msgs._ptr(g[k]) for k in NAMES))
    wsb = msgs.ms_raster_bwd_views_workspace_bytes(sc.n, len(views))
    wsd = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    msgs.ms_raster_bwd_views(ds.struct, views, grads, 0, msgs._ptr(wsd), wsb)
    torch.cuda.synchronize()
    gg = {k: g[k].cpu().numpy().astype(np.float64) for k in NAMES}
    go = {k: 0.0 for k in NAMES}
    for cam, w in zip(cams, ws_):
        fp = oracle.footprints(sc, cam, "all_levels")
        off, idx = oracle.tile_lists(fp, cam)
        g1 = oracle.grad64(sc, cam, off, idx, w)
        go = {k: go[k] + g1[k] for k in NAMES}
    compare(gg, go)
    # the two passes run by themselves, one after the other (the raster
    # pass's 2D gradients stay in the workspace for the projection pass)
    for k in NAMES:
        g[k].fill_(float("nan"))
    msgs.ms_raster_bwd_views(ds.struct, views, grads, msgs.MS_BWD_RASTER_PASS,
                             msgs._ptr(wsd), wsb)
    msgs.ms_raster_bwd_views(ds.struct, views, grads, msgs.MS_BWD_PROJECT_PASS,
                             msgs._ptr(wsd), wsb)
    torch.cuda.synchronize()
    compare({k: g[k].cpu().numpy().astype(np.float64) for k in NAMES}, go)
    with pytest.raises(msgs.MsError):
        msgs.ms_raster_bwd_views(ds.struct, views, grads, 8, msgs._ptr(wsd), wsb)


def test_autograd_views_equals_sum_of_single_views():
    torch = require_cuda()
    dev = torch.device("cuda")
    sc = inputs.tiny_scene(n=300, seed=13, sh_degree=2, extent=0.8)
    cams = [inputs.config1_camera(64, 64), inputs.config1_camera(32, 32)]
    level = torch.tensor(sc.level, device=dev)
    smax = torch.tensor(sc.s_max, device=dev)
    smin = torch.tensor(sc.s_min, device=dev)
    rng = np.random.default_rng(13)
    ws_ = [torch.tensor(rng.standard_normal((3, c.height, c.width)), dtype=torch.float32,
                        device=dev) for c in cams]

    def fresh():
        return {k: torch.tensor(getattr(sc, k), device=dev, requires_grad=True) for k in NAMES}
    p1 = fresh()
    frames = [ag.Frame(sc.n, c, 64 * sc.n, device=dev) for c in cams]
    imgs = ag.render_views(p1, level, smax, smin, 1, sc.sh_degree, frames, "all_levels")
    sum(((im * w).sum() for im, w in zip(imgs, ws_)), torch.zeros((), device=dev)).backward()
    p2 = fresh()
    total = torch.zeros((), device=dev)
    for c, w in zip(cams, ws_):
        im = ag.render(p2, level, smax, smin, 1, sc.sh_degree, ag.Frame(sc.n, c, 64 * sc.n,
                                                                       device=dev), "all_levels")
        total = total + (im * w).sum()
    total.backward()
    torch.cuda.synchronize()
    for k in NAMES:
        a, b = p1[k].grad.cpu().numpy(), p2[k].grad.cpu().numpy()
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-5 * np.abs(b).max())
