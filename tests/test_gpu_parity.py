"""Parity of the CUDA path (through the C ABI) with the oracle.

Footprints, selection masks and per-tile sorted index lists must be
bit-exact; images within 2e-4 max abs per channel on pixels where no
Gaussian sits on the alpha threshold (the oracle flags those)."""
import numpy as np
import pytest

import oracle
import paper_2311_17089_gb300 as msgs
from paper_2311_17089_gb300 import inputs

from gpu_util import (assert_footprints_equal, assert_image_close, assert_lists_equal,
                      calibrated, gpu_frame, mask_bits, require_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    return require_cuda()


@pytest.fixture(scope="module")
def ms_scene_50k():
    sc = inputs.multiscale_scene(n=50_000, seed=0)
    return calibrated(sc, inputs.orbit_cameras(8, seed=1, radius=25.0))


def test_scene_prepare_matches_oracle(cuda):
    sc = inputs.multiscale_scene(n=200_000, seed=3)
    ds = msgs.DeviceScene(sc)
    cuda.cuda.synchronize()
    scale, lnop = oracle.prepare(sc)
    np.testing.assert_array_equal(ds.scale.cpu().numpy(), scale)
    np.testing.assert_array_equal(ds.lnop.cpu().numpy(), lnop)


# "tile@K": the tile kernel on at most K CTAs per SM (ms_raster_ex2), which
# also changes the frame's segmentation; "auto" launches both the tile and
# the list kernel for frames of 1-4x as many tiles as SMs and lets the
# device pick one
STRATEGIES = ["auto", "tile", "tile@1", "tile@2", "list", "group8", "group16", "group32"]


@pytest.mark.parametrize("strategy", STRATEGIES)
@pytest.mark.parametrize("mode", ["all_levels", "selective"])
def test_single_level_config_full_parity(cuda, mode, strategy):
    """10k single-level Gaussians, 256x256 (16x16 tiles), with either
    raster kernel."""
    sc = inputs.single_level_scene()
    cam = inputs.config1_camera()
    g = gpu_frame(sc, cam, mode, strategy=strategy)
    o = oracle.render(sc, cam, mode)
    assert_footprints_equal(g, o["fp"], sc, cam)
    assert_lists_equal(g, o["offsets"], o["idx"])
    err, flagged = assert_image_close(g, o)
    assert flagged < 0.01 * cam.width * cam.height


@pytest.mark.parametrize("strategy", STRATEGIES)
@pytest.mark.parametrize("scale", [1, 2, 4, 8, 16, 32, 64, 128])
@pytest.mark.parametrize("mode", ["selective", "all_levels", "filter_small"])
def test_multiscale_all_scales(cuda, ms_scene_50k, mode, scale, strategy):
    """50k-Gaussian 4-level scene at every evaluation scale of 1256x832
    (ragged right-hand tiles at most scales), with either raster kernel."""
    sc = ms_scene_50k
    cam = inputs.downscale(inputs.config2_camera(), scale)
    g = gpu_frame(sc, cam, mode, strategy=strategy)
    o = oracle.render(sc, cam, mode)
    assert_footprints_equal(g, o["fp"], sc, cam)
    assert_lists_equal(g, o["offsets"], o["idx"])
    assert_image_close(g, o)


def test_selective_differs_from_all_levels_and_skips_levels(cuda, ms_scene_50k):
    """Sanity of the workload: at 1x most coarse Gaussians are filtered,
    at 64x most fine ones are."""
    sc = ms_scene_50k
    for s, dropped_level in ((1, 4), (64, 1)):
        cam = inputs.downscale(inputs.config2_camera(), s)
        g = gpu_frame(sc, cam, "selective")
        sel = mask_bits(g["mask"], sc.n)
        lv = sc.level == dropped_level
        assert sel[lv].mean() < 0.5


def test_select_entry_point_matches_project_mask(cuda, ms_scene_50k):
    torch = cuda
    sc = ms_scene_50k
    cam = inputs.downscale(inputs.config2_camera(), 4)
    ds = msgs.DeviceScene(sc)
    r = msgs.Renderer(sc.n, cam.tiles_x * cam.tiles_y, 16 * sc.n)
    for mode in ("selective", "all_levels", "filter_small"):
        msgs.ms_project(ds.struct, msgs.camera_struct(cam), msgs.MODES[mode], r.proj)
        m2 = torch.empty_like(r.mask)
        msgs.ms_select(ds.struct, msgs._ptr(r.cover), msgs.MODES[mode], msgs._ptr(m2))
        torch.cuda.synchronize()
        assert torch.equal(r.mask, m2)


def test_update_range_matches_oracle(cuda):
    """Device UpdateRange over a calibration sequence (8 cameras x 4 levels at
    each level's creation scale) equals the oracle's, bit for bit."""
    sc = inputs.multiscale_scene(n=100_000, seed=5)
    cams = inputs.orbit_cameras(8, seed=2, radius=25.0)
    ds = msgs.DeviceScene(sc)
    ds.calibrate(cams)
    want = oracle.calibrate(sc.copy(), cams)
    np.testing.assert_array_equal(ds.s_max.cpu().numpy(), want.s_max)
    np.testing.assert_array_equal(ds.s_min.cpu().numpy(), want.s_min)


def test_full_size_multiscale_sampled(cuda):
    """1M Gaussians (700k/200k/70k/30k) at 1256x832, the launch shape the
    benchmark times: every footprint and every tile list bit-exact; the
    image on 48 sampled tiles plus the longest list's tile."""
    sc = inputs.multiscale_scene(n=1_000_000, seed=0)
    sc = calibrated(sc, inputs.orbit_cameras(8, seed=1, radius=25.0))
    rng = np.random.default_rng(0)
    for mode in ("selective", "all_levels"):
        # 4x: 260 tiles, where the device picks the list kernel for the
        # selective frame (short lists) and the tile kernel at all levels
        for s in (1, 4, 16, 128):
            cam = inputs.downscale(inputs.config2_camera(), s)
            g = gpu_frame(sc, cam, mode)
            fp = oracle.footprints(sc, cam, mode)
            assert_footprints_equal(g, fp, sc, cam)
            off, idx = oracle.tile_lists(fp, cam)
            assert_lists_equal(g, off, idx)
            ntiles = cam.tiles_x * cam.tiles_y
            tiles = sorted(set(rng.choice(ntiles, min(48, ntiles), replace=False).tolist()
                               + [int(np.argmax(np.diff(off)))]))
            o = oracle.render(sc, cam, mode, tiles=tiles)
            assert_image_close(g, o, tiles=tiles, cam=cam)


def test_full_size_near_far_sampled(cuda):
    """3M Gaussians: a dense unit ball and a sparse shell of radius 50
    (the near/far stress workload), cameras on an orbit at radii from 2
    to 60, at 8x and 64x of 1256x832: every footprint and tile list
    bit-exact; the image on sampled tiles plus the longest list's tile."""
    sc = inputs.near_far_scene(n=3_000_000, seed=0)
    radii = np.geomspace(2.0, 60.0, 32)
    cams = inputs.orbit_cameras(32, seed=3, radius=radii)
    sc = calibrated(sc, cams[::8])
    rng = np.random.default_rng(1)
    ds = msgs.DeviceScene(sc)
    for k in (0, 15, 31):
        for s in (8, 64):
            cam = inputs.downscale(cams[k], s)
            g = gpu_frame(sc, cam, "selective", ds=ds)
            fp = oracle.footprints(sc, cam, "selective")
            assert_footprints_equal(g, fp, sc, cam)
            off, idx = oracle.tile_lists(fp, cam)
            assert_lists_equal(g, off, idx)
            ntiles = cam.tiles_x * cam.tiles_y
            tiles = sorted(set(rng.choice(ntiles, min(12, ntiles), replace=False).tolist()
                               + [int(np.argmax(np.diff(off)))]))
            o = oracle.render(sc, cam, "selective", tiles=tiles)
            assert_image_close(g, o, tiles=tiles, cam=cam)


# ------------------------------------------------------------- edge cases

@pytest.mark.parametrize("strategy", STRATEGIES)
def test_empty_scene(cuda, strategy):
    sc = inputs.single_level_scene(n=0)
    cam = inputs.config1_camera(40, 24)
    cam.bg[:] = [0.25, 0.5, 1.0]
    g = gpu_frame(sc, cam, "selective", strategy=strategy)
    assert g["D"] == 0
    np.testing.assert_array_equal(g["image"], np.broadcast_to(cam.bg[:, None, None], (3, 24, 40)))
    assert np.all(g["final_t"] == 1.0) and np.all(g["n_contrib"] == 0)


def test_everything_culled(cuda):
    sc = inputs.single_level_scene(n=5000)
    cam = inputs.pinhole((0, 0, -3), (0, 0, -6), (0, -1, 0), 64, 64, 60.0)  # looks away
    g = gpu_frame(sc, cam, "all_levels")
    o = oracle.render(sc, cam, "all_levels")
    assert g["D"] == 0 and len(o["idx"]) == 0
    assert_footprints_equal(g, o["fp"], sc, cam)
    assert np.all(g["image"] == 0.0)


@pytest.mark.parametrize("strategy", STRATEGIES)
@pytest.mark.parametrize("wh", [(1, 1), (33, 17), (16, 16), (17, 1), (300, 7)])
def test_ragged_sizes(cuda, wh, strategy):
    sc = inputs.single_level_scene(n=3000, seed=4)
    cam = inputs.config1_camera(*wh)
    cam.bg[:] = [0.1, 0.2, 0.3]
    g = gpu_frame(sc, cam, "all_levels", strategy=strategy)
    o = oracle.render(sc, cam, "all_levels")
    assert_footprints_equal(g, o["fp"], sc, cam)
    assert_lists_equal(g, o["offsets"], o["idx"])
    assert_image_close(g, o)


def test_degenerate_and_nonfinite_inputs(cuda):
    sc = inputs.single_level_scene(n=2000, seed=6)
    sc.quat[0:10] = 0.0                       # no rotation -> invalid
    sc.mean[10:20, 0] = np.nan                # NaN centre -> invalid
    sc.log_scale[20:30] = -30.0               # vanishing scale
    sc.log_scale[30:35] = 30.0                # enormous scale
    sc.opacity[35:45] = 1.0 / 255.0           # no level set
    sc.opacity[45:50] = 1e-6
    sc.mean[50:60, 2] = -3.0                  # exactly at the camera plane
    cam = inputs.config1_camera(96, 80)
    g = gpu_frame(sc, cam, "all_levels")
    o = oracle.render(sc, cam, "all_levels")
    assert_footprints_equal(g, o["fp"], sc, cam)
    assert not o["fp"]["valid"][:20].any()
    assert_lists_equal(g, o["offsets"], o["idx"])
    assert_image_close(g, o)


def test_depth_ties_order_by_index(cuda):
    """Many Gaussians on one depth plane: lists order ties by index."""
    sc = inputs.single_level_scene(n=20_000, seed=8)
    sc.mean[:, 2] = np.round(sc.mean[:, 2] * 4) / 4   # 9 depth planes
    cam = inputs.config1_camera(128, 96)
    g = gpu_frame(sc, cam, "all_levels")
    o = oracle.render(sc, cam, "all_levels")
    assert_lists_equal(g, o["offsets"], o["idx"])
    assert_image_close(g, o)


def test_huge_gaussian_covers_every_tile(cuda):
    sc = inputs.single_level_scene(n=200, seed=9)
    sc.log_scale[7] = 1.0
    sc.mean[7] = 0.0
    cam = inputs.config1_camera(256, 192)
    g = gpu_frame(sc, cam, "all_levels")
    o = oracle.render(sc, cam, "all_levels")
    assert o["fp"]["ntiles"][7] == cam.tiles_x * cam.tiles_y
    assert_lists_equal(g, o["offsets"], o["idx"])
    assert_image_close(g, o)


def test_capacity_overflow_reported_then_retry(cuda):
    torch = cuda
    sc = inputs.single_level_scene(n=10_000)
    cam = inputs.config1_camera()
    ds = msgs.DeviceScene(sc)
    r = msgs.Renderer(sc.n, cam.tiles_x * cam.tiles_y, 1000)
    r.render(ds, cam, "all_levels")
    rc, d, _ = msgs.ms_bin_counts(r.bins)
    assert rc == msgs.MS_ERR_CAPACITY and d > 1000
    o = oracle.render(sc, cam, "all_levels")
    assert d == len(o["idx"])
    g = gpu_frame(sc, cam, "all_levels", cap=d)
    assert_lists_equal(g, o["offsets"], o["idx"])


@pytest.mark.parametrize("strategy", STRATEGIES)
@pytest.mark.parametrize("wh,n,op", [((16, 16), 6000, (0.008, 0.014)),
                                     ((48, 32), 9000, (0.008, 0.014)),
                                     ((16, 16), 1500, (0.0050, 0.0058))])
def test_long_lists_split_across_ctas(cuda, wh, n, op, strategy):
    """Thousands of faint, wide Gaussians on few tiles.  The tile kernel
    splits the lists into segments blended by different CTAs; the list
    kernel walks each pixel's whole list across the lanes of one warp.
    With opacity ~0.01 every pixel's T falls about 1% per Gaussian and it
    terminates inside a later segment; with opacity ~0.005 over 1500
    entries no pixel terminates.  Both must reproduce the sequential
    blend."""
    rng = np.random.default_rng(n)
    mean = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.4, 0.4, n),
                     rng.uniform(-1.0, 1.0, n)], 1).astype(np.float32)
    log_scale = rng.normal(np.log(6.0), 0.05, (n, 3)).astype(np.float32)
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    opacity = rng.uniform(op[0], op[1], n).astype(np.float32)
    color = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    sc = inputs.Scene(mean, log_scale, quat, opacity, color, np.ones(n, np.uint8), 1, -1,
                      np.zeros(n, np.float32), np.full(n, np.inf, np.float32))
    cam = inputs.config1_camera(*wh)
    g = gpu_frame(sc, cam, "all_levels", strategy=strategy)
    o = oracle.render(sc, cam, "all_levels")
    assert_lists_equal(g, o["offsets"], o["idx"])
    assert np.diff(o["offsets"]).max() > 1024
    if op[0] > 0.007:
        assert (o["n_contrib"] > 600).all() and (o["final_t"] < 1.1e-2).all()
    else:
        assert (o["n_contrib"] == n).all()
    assert_image_close(g, o)


def deep_lists_scene(seed=31, nb=40_000):
    """A 48x32 frame whose tile lists hold more than 4096 entries: nb (40k)
    faint Gaussians about 2 px wide spread over the whole view (each pixel
    sees a few percent of its tile's list, so most pixels never terminate
    and blend entries past 4096), and 400 large, fairly opaque ones in
    front of the left half (those pixels terminate within the first few
    dozen entries)."""
    rng = np.random.default_rng(seed)
    nf = 400
    n = nf + nb
    mean = np.empty((n, 3), np.float32)
    mean[:nf] = np.stack([rng.uniform(-0.75, 0.0, nf), rng.uniform(-0.5, 0.5, nf),
                          rng.uniform(-1.8, -1.6, nf)], 1)
    mean[nf:] = np.stack([rng.uniform(-1.8, 1.8, nb), rng.uniform(-1.2, 1.2, nb),
                          rng.uniform(-0.3, 0.3, nb)], 1)
    log_scale = np.empty((n, 3), np.float32)
    log_scale[:nf] = rng.normal(np.log(0.08), 0.1, (nf, 3))
    log_scale[nf:] = rng.normal(np.log(0.03), 0.1, (nb, 3))
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    opacity = np.concatenate([rng.uniform(0.5, 0.9, nf), rng.uniform(0.01, 0.03, nb)]).astype(np.float32)
    color = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    return inputs.Scene(mean, log_scale, quat, opacity, color, np.ones(n, np.uint8), 1, -1,
                        np.zeros(n, np.float32), np.full(n, np.inf, np.float32))


@pytest.mark.parametrize("strategy", STRATEGIES)
def test_long_lists_early_and_deep_pixels(cuda, strategy):
    """Six tiles whose lists hold 7.5k-8.3k entries: about half of the
    pixels terminate within the first few dozen entries, the other half
    blend entries past 4096 and mostly never terminate (the list kernel's
    slowest case: one warp walks such a pixel's whole list)."""
    sc = deep_lists_scene()
    cam = inputs.config1_camera(48, 32)
    o = oracle.render(sc, cam, "all_levels")
    assert np.diff(o["offsets"]).min() > 4096 + 1024
    early = (o["final_t"] < 1e-3) & (o["n_contrib"] < 2048)
    deep = o["n_contrib"] > 4096 + 512
    assert early.mean() > 0.2 and deep.mean() > 0.2, (early.mean(), deep.mean())
    g = gpu_frame(sc, cam, "all_levels", strategy=strategy)
    assert_lists_equal(g, o["offsets"], o["idx"])
    assert_image_close(g, o)


@pytest.mark.parametrize("strategy", ["auto", "list"])
def test_lists_past_the_mask_prefix(cuda, strategy):
    """Lists of 19k-22k entries, with deep pixels blending entries past the
    first 16384 of their tile's list: the list kernel's mask pass covers
    only that prefix, and past it each thread forms its entries' half-row
    masks itself."""
    sc = deep_lists_scene(seed=35, nb=110_000)
    cam = inputs.config1_camera(48, 32)
    o = oracle.render(sc, cam, "all_levels")
    assert np.diff(o["offsets"]).min() > 16384 + 1024
    assert (o["n_contrib"] > 16384 + 512).mean() > 0.2
    g = gpu_frame(sc, cam, "all_levels", strategy=strategy)
    assert_lists_equal(g, o["offsets"], o["idx"])
    assert_image_close(g, o)


def test_one_long_list_among_many_tiles_and_overflow(cuda):
    """A 320-tile frame where one tile lists ~30k Gaussians among many short
    lists: lists bit-exact and image within tolerance; a capacity far below
    D reports the exact D and the retry matches."""
    rng = np.random.default_rng(21)
    n = 30_000
    sc = inputs.single_level_scene(n=n, seed=21)
    # most Gaussians packed around one point (one tile), the rest spread out
    sc.mean[: n - 2000] = (rng.normal(0.0, 0.01, (n - 2000, 3)) + [0.05, 0.05, 0.0]).astype(np.float32)
    sc.log_scale[: n - 2000] = rng.normal(-4.0, 0.3, (n - 2000, 3)).astype(np.float32)
    cam = inputs.config1_camera(320, 256)
    fp = oracle.footprints(sc, cam, "all_levels")
    off, idx = oracle.tile_lists(fp, cam)
    assert cam.tiles_x * cam.tiles_y >= 200 and np.diff(off).max() > 3 * 8192
    g = gpu_frame(sc, cam, "all_levels", cap=1000)   # overflows first, then retries
    assert g["D"] == len(idx)
    assert_lists_equal(g, off, idx)
    o = oracle.render(sc, cam, "all_levels")
    assert_image_close(g, o, cam=cam)


def test_scene_prepare_bit_exact_many_values(cuda):
    """exp(log_scale) and ln(255 opacity) rounded to float, on 4M values
    across the float range the scenes use and its edges (the device
    evaluates them in float-float with an FP64 decision near midpoints)."""
    import torch
    rng = np.random.default_rng(17)
    m = 4_000_000
    ls = np.concatenate([rng.uniform(-12.0, 6.0, m // 2), rng.normal(-3.5, 2.0, m // 4),
                         rng.uniform(-79.9, 79.9, m // 4)]).astype(np.float32)
    op = np.concatenate([rng.uniform(0.0, 1.0, m // 2), 1.0 / (1.0 + np.exp(-rng.normal(0, 3, m // 4))),
                         10.0 ** rng.uniform(-30, 0, m // 4)]).astype(np.float32)
    tiny = np.float32(1.0 / 255.0)
    edges_ls = np.array([0.0, -0.0, 1e-30, -1e-30, 79.99, -79.99, 80.0, -80.0, 88.0, -87.0,
                         100.0, np.inf, -np.inf, np.nan], np.float32)
    edges_op = np.array([1.0, 0.5, tiny, np.nextafter(tiny, np.float32(1)),
                         np.nextafter(tiny, np.float32(0)), 1e-6, 1e-30, 1e-35, 0.0, -0.5,
                         np.inf, np.nan, 3.0, 1e31], np.float32)
    ls = np.concatenate([ls, edges_ls])
    op = np.concatenate([op, edges_op])
    n = len(ls) // 3 * 3
    sc = inputs.single_level_scene(n=n // 3, seed=0)
    sc.log_scale = ls[:n].reshape(-1, 3)
    sc.opacity = op[: n // 3]
    want_scale, want_lnop = oracle.prepare(sc)
    dev = torch.device("cuda")
    lsd = torch.tensor(sc.log_scale, device=dev)
    opd = torch.tensor(sc.opacity, device=dev)
    scale = torch.empty_like(lsd)
    lnop = torch.empty_like(opd)
    st = msgs.ms_scene_t(sc.n, 1, -1, 1, msgs._ptr(lsd), 1, msgs._ptr(opd), 1, 1, 1, 1,
                         msgs._ptr(scale), msgs._ptr(lnop))
    msgs.ms_scene_prepare(st)
    torch.cuda.synchronize()
    for got, want in ((scale.cpu().numpy(), want_scale), (lnop.cpu().numpy(), want_lnop)):
        nan = np.isnan(want)          # NaN payloads may differ; positions may not
        np.testing.assert_array_equal(np.isnan(got), nan)
        np.testing.assert_array_equal(got[~nan].view(np.uint32), want[~nan].view(np.uint32))


def band_scene(seed=41, n=36_000):
    """36k faint Gaussians about 10 px wide over a 320x240 frame (300
    tiles, 1.2k-2.6k entries per tile list): a frame with 1-4x as many
    tiles as SMs and a mean list length of 1024-8192, which ms_raster
    (MS_RASTER_AUTO) hands to the list kernel on the device."""
    rng = np.random.default_rng(seed)
    mean = np.stack([rng.uniform(-1.9, 1.9, n), rng.uniform(-1.4, 1.4, n),
                     rng.uniform(-0.5, 0.5, n)], 1).astype(np.float32)
    log_scale = rng.normal(np.log(0.12), 0.15, (n, 3)).astype(np.float32)
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    opacity = rng.uniform(0.02, 0.10, n).astype(np.float32)
    color = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    return inputs.Scene(mean, log_scale, quat, opacity, color, np.ones(n, np.uint8), 1, -1,
                        np.zeros(n, np.float32), np.full(n, np.inf, np.float32))


@pytest.mark.parametrize("strategy", ["auto", "tile", "list"])
def test_band_frame(cuda, strategy):
    """The frame where ms_raster launches both blend kernels and the device
    picks one: the same lists and image whichever blends it."""
    sc = band_scene()
    cam = inputs.config1_camera(320, 240)
    o = oracle.render(sc, cam, "all_levels")
    tiles = cam.tiles_x * cam.tiles_y
    assert 152 <= tiles < 4 * 152
    assert 1024 * tiles <= len(o["idx"]) <= 8192 * tiles
    g = gpu_frame(sc, cam, "all_levels", strategy=strategy)
    assert_lists_equal(g, o["offsets"], o["idx"])
    assert_image_close(g, o)
