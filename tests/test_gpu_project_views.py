"""ms_project_views: several cameras projected in one pass must write, for
every view, exactly what ms_project writes for that camera alone (the
bit-exact footprint contract), whatever the number of views, the mode, the
mix of camera centres (views with a shared centre share the SH colour) and
the invalid Gaussians; and the footprints of a view match the oracle's.
Frames rendered by render_views equal frames rendered one by one."""
import numpy as np
import pytest

import oracle
import paper_2311_17089_gb300 as msgs
from paper_2311_17089_gb300 import inputs

from gpu_util import assert_footprints_equal, calibrated, require_cuda

pytestmark = pytest.mark.gpu

BUFFERS = ("rec", "rect", "n_tiles", "depth", "cover", "mask", "stats")


@pytest.fixture(scope="module")
def cuda():
    return require_cuda()


@pytest.fixture(scope="module")
def ms_scene_50k():
    sc = inputs.multiscale_scene(n=50_000, seed=0)
    return calibrated(sc, inputs.orbit_cameras(8, seed=1, radius=25.0))


def degenerate_scene():
    """A ragged count (not a multiple of the 256-Gaussian chunk) with
    invalid Gaussians of every kind."""
    sc = inputs.single_level_scene(n=3001, seed=6)
    sc.quat[0:10] = 0.0
    sc.mean[10:20, 0] = np.nan
    sc.log_scale[20:30] = -30.0
    sc.log_scale[30:35] = 30.0
    sc.opacity[35:45] = 1.0 / 255.0
    sc.mean[50:60, 2] = -3.0
    return sc


def renderers(sc, cams):
    rs = [msgs.Renderer(sc.n, c.tiles_x * c.tiles_y, 16 * sc.n + 4096) for c in cams]
    for r in rs:  # unlisted entries are not written: start from zeros on both sides
        for b in BUFFERS:
            getattr(r, b).zero_()
    return rs


def project_both(torch, sc, cams, mode):
    ds = msgs.DeviceScene(sc)
    alone, joint = renderers(sc, cams), renderers(sc, cams)
    m = msgs.MODES[mode]
    for r, c in zip(alone, cams):
        msgs.ms_project(ds.struct, msgs.camera_struct(c), m, r.proj)
    msgs.ms_project_views(ds.struct, [msgs.camera_struct(c) for c in cams], m,
                          [r.proj for r in joint])
    torch.cuda.synchronize()
    return alone, joint


def assert_views_equal(alone, joint):
    for v, (a, j) in enumerate(zip(alone, joint)):
        for b in BUFFERS:
            assert getattr(a, b).equal(getattr(j, b)), (v, b)


def shared_centre_cams():
    return [inputs.downscale(inputs.config2_camera(), s) for s in inputs.SCALES]


def mixed_cams():
    """Centres A, B, A, C, B, A: a Gaussian's colour is evaluated again
    whenever the centre changes and reused when it repeats."""
    a, b, c = inputs.orbit_cameras(3, seed=4, radius=25.0, width=400, height=300)
    return [a, b, inputs.downscale(a, 2), c, inputs.downscale(b, 4), inputs.downscale(a, 8)]


@pytest.mark.parametrize("mode", ["selective", "all_levels", "filter_small"])
def test_eight_views_shared_centre_equal_single_views(cuda, ms_scene_50k, mode):
    alone, joint = project_both(cuda, ms_scene_50k, shared_centre_cams(), mode)
    assert_views_equal(alone, joint)
    assert all(int(r.n_tiles.count_nonzero()) > 0 for r in joint)


@pytest.mark.parametrize("n_views", [1, 2, 3, 6])
def test_mixed_centres_any_view_count(cuda, ms_scene_50k, n_views):
    cams = mixed_cams()[:n_views]
    alone, joint = project_both(cuda, ms_scene_50k, cams, "selective")
    assert_views_equal(alone, joint)


def pruned_both(torch, sc, cams, ds=None):
    """Selective views of one pose without coverage output (the launch that
    leaves out footprints its coverage bound rules out) against each camera
    projected alone."""
    ds = ds or msgs.DeviceScene(sc)
    n = sc.n

    def rs():
        out = [msgs.Renderer(n, c.tiles_x * c.tiles_y, 16, with_cover=False) for c in cams]
        for r in out:
            for b in ("rec", "rect", "n_tiles", "depth", "mask", "stats"):
                getattr(r, b).zero_()
        return out
    alone, joint = rs(), rs()
    m = msgs.MODES["selective"]
    for r, c in zip(alone, cams):
        msgs.ms_project(ds.struct, msgs.camera_struct(c), m, r.proj)
    msgs.ms_project_views(ds.struct, [msgs.camera_struct(c) for c in cams], m,
                          [r.proj for r in joint])
    torch.cuda.synchronize()
    pruned = 0
    for v, (a, j) in enumerate(zip(alone, joint)):
        for b in ("rec", "n_tiles", "depth", "mask", "stats"):
            assert getattr(a, b).equal(getattr(j, b)), (v, b)
        listed = a.n_tiles[:n] != 0
        ra, rj = a.rect.view(-1, 2)[:n], j.rect.view(-1, 2)[:n]
        assert ra[listed].equal(rj[listed]), v
        # a pair left out holds the empty rectangle
        empty = (rj[:, 0] == 0) & (rj[:, 1] == -1)
        assert bool((empty | (ra == rj).all(1)).all()), v
        pruned += int((~(ra == rj).all(1)).sum())
    return pruned


def test_pruned_views_equal_single_views(cuda, ms_scene_50k):
    """The eight scales of one pose: the views' footprints the coverage
    bound rules out are left out, and every list, record, mask and stat
    still equals the camera's own ms_project bit for bit."""
    pruned = pruned_both(cuda, ms_scene_50k, shared_centre_cams())
    assert pruned > 10_000


def test_pruned_views_on_the_1M_sweep(cuda):
    """The 1M four-level scene with its calibrated ranges (many Gaussians
    near a range's edge) at the eight scales of the bench sweep."""
    sc = inputs.multiscale_scene(n=1_000_000, seed=0)
    ds = msgs.DeviceScene(sc)
    ds.calibrate(inputs.orbit_cameras(8, seed=1, radius=25.0))
    cams = [inputs.downscale(inputs.config2_camera(), s) for s in inputs.SCALES]
    assert pruned_both(cuda, sc, cams, ds) > 1_000_000


def test_pruned_views_at_the_range_edges(cuda):
    """Ranges placed on the selection thresholds of Eq. 6: every Gaussian's
    s_max puts S / s_max within a few ulps of 1.5 in one view and its s_min
    puts S / s_min within a few ulps of 0.5 in another, and a third of the
    Gaussians are needles (one axis 400x shorter, so their 2D covariance is
    badly conditioned).  The bound must leave out no footprint that the
    exact comparison would select."""
    torch = cuda
    sc = inputs.multiscale_scene(n=20_000, seed=3)
    sc.log_scale[::3, 2] -= 6.0
    ds = msgs.DeviceScene(sc)
    cams = shared_centre_cams()
    n = sc.n
    rs = [msgs.Renderer(n, c.tiles_x * c.tiles_y, 16) for c in cams]
    msgs.ms_project_views(ds.struct, [msgs.camera_struct(c) for c in cams],
                          msgs.MODES["all_levels"], [r.proj for r in rs])
    torch.cuda.synchronize()
    S = torch.stack([r.cover[:n] for r in rs], 1).double()          # n x 8, exact FP32 S
    rng = np.random.default_rng(11)
    va = torch.from_numpy(rng.integers(0, 4, n)).cuda()             # views 1x .. 8x
    vb = torch.from_numpy(rng.integers(3, 8, n)).cuda()             # views 8x .. 128x
    ka = torch.from_numpy(rng.integers(-3, 4, n).astype(np.float64)).cuda()
    kb = torch.from_numpy(rng.integers(-3, 4, n).astype(np.float64)).cuda()
    u = 2.0 ** -24
    sa = S.gather(1, va[:, None])[:, 0]
    sb = S.gather(1, vb[:, None])[:, 0]
    smax = sa / 1.5 * (1.0 + ka * u)
    smin = sb / 0.5 * (1.0 + kb * u)
    ok = (sa > 0) & (sb > 0)
    ds.s_max[:n] = torch.where(ok, smax, torch.ones_like(smax)).float()
    ds.s_min[:n] = torch.where(ok, smin, torch.ones_like(smin)).float()
    assert pruned_both(torch, sc, cams, ds) > 1000


def test_pruned_views_ragged_invalid(cuda):
    sc = degenerate_scene()
    sc.level[:] = np.arange(sc.n) % 3 + 1
    sc.n_levels = 3
    ds = msgs.DeviceScene(sc)
    ds.calibrate([inputs.config1_camera()])
    cams = [inputs.downscale(inputs.config1_camera(400, 300), s) for s in (1, 2, 4, 8, 16)]
    pruned_both(cuda, sc, cams, ds)


def test_invalid_gaussians_and_ragged_chunk(cuda):
    sc = degenerate_scene()
    cams = [inputs.config1_camera(96, 80), inputs.config1_camera(48, 40),
            inputs.config1_camera(400, 300)]
    alone, joint = project_both(cuda, sc, cams, "all_levels")
    assert_views_equal(alone, joint)
    assert int(joint[0].n_tiles[:20].count_nonzero()) == 0


def test_views_match_oracle_footprints(cuda, ms_scene_50k):
    sc = ms_scene_50k
    cams = mixed_cams()
    _, joint = project_both(cuda, sc, cams, "selective")
    n = sc.n
    for r, cam in zip(joint, cams):
        g = dict(n_tiles=r.n_tiles.cpu().numpy().view(np.uint32)[:n],
                 depth=r.depth.cpu().numpy().view(np.uint32)[:n],
                 rect=r.rect.cpu().numpy().view(np.uint32).reshape(-1, 2)[:n],
                 cover=r.cover.cpu().numpy()[:n], mask=r.mask.cpu().numpy().view(np.uint32),
                 rec=r.rec.cpu().numpy().reshape(-1, 12)[:n])
        assert_footprints_equal(g, oracle.footprints(sc, cam, "selective"), sc, cam)


def test_render_views_equals_frames_rendered_alone(cuda, ms_scene_50k):
    torch = cuda
    sc = ms_scene_50k
    cams = shared_centre_cams() + mixed_cams()[:3]  # 11 frames: two projection passes
    ds = msgs.DeviceScene(sc)
    alone = [msgs.Renderer(sc.n, c.tiles_x * c.tiles_y, 16 * sc.n) for c in cams]
    joint = [msgs.Renderer(sc.n, c.tiles_x * c.tiles_y, 16 * sc.n) for c in cams]
    want = [r.render(ds, c, "selective") for r, c in zip(alone, cams)]
    streams = [torch.cuda.Stream() for _ in cams]
    got = msgs.render_views(ds, joint, cams, "selective", streams=streams)
    torch.cuda.synchronize()
    for r in alone + joint:
        r.check()
    for v, (w, g) in enumerate(zip(want, got)):
        for a, b in zip(w, g):
            assert a.equal(b), v


@pytest.mark.parametrize("split", [False, True])
def test_render_views_sharing_the_sms_equals_frames_rendered_alone(cuda, ms_scene_50k, split):
    """render_views with share_sms: the frames the tile kernel blends run on
    share_ctas_per_sm() CTAs per SM and the others start once those have
    binned; every frame equals the frame rendered alone with the same
    kernel and CTA count, bit for bit (also from a shared, split depth
    order)."""
    torch = cuda
    sc = ms_scene_50k
    cams = shared_centre_cams()
    ds = msgs.DeviceScene(sc)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    alone = [msgs.Renderer(sc.n, c.tiles_x * c.tiles_y, 16 * sc.n) for c in cams]
    tmax = max(c.tiles_x * c.tiles_y for c in cams)
    want = [r.render(ds, c, "selective",
                     max_ctas_per_sm=(msgs.share_ctas_per_sm(c.tiles_x * c.tiles_y, tmax)
                                      if c.tiles_x * c.tiles_y >= sms else 0))
            for r, c in zip(alone, cams)]
    joint = [msgs.Renderer(sc.n, c.tiles_x * c.tiles_y, 16 * sc.n, with_cover=False)
             for c in cams]
    streams = [torch.cuda.Stream() for _ in cams]
    order = msgs.DepthOrder(sc.n, split_views=len(cams)) if split else None
    got = msgs.render_views(ds, joint, cams, "selective", streams=streams, order=order,
                            share_sms=True)
    torch.cuda.synchronize()
    assert sum(c.tiles_x * c.tiles_y >= sms for c in cams) >= 2
    for r in alone + joint:
        r.check()
    for v, (w, g) in enumerate(zip(want, got)):
        for a, b in zip(w, g):
            assert a.equal(b), v


@pytest.mark.parametrize("mode", ["all_levels", "selective"])
def test_histogram_flush_on_a_30M_scene(cuda, mode):
    """30M Gaussians: with two views (456 CTAs of 256 threads) every CTA
    processes more than 255 chunks, so its 16-bit digit counts are flushed
    mid-launch; one view (608 CTAs) never flushes early.  Counters,
    histograms and footprints still agree bit for bit, in both the plain
    multi-view launch and the pruning one (one level: nothing is left
    out, every pair is packed)."""
    torch = cuda
    sc = inputs.single_level_scene(n=30_000_000, seed=9)
    ds = msgs.DeviceScene(sc)
    n = sc.n
    cams = [inputs.config1_camera(96, 80), inputs.config1_camera(40, 24)]

    def proj():
        t = dict(rec=torch.zeros(n * 12, dtype=torch.float32, device="cuda"),
                 rect=torch.zeros(n * 2, dtype=torch.int32, device="cuda"),
                 n_tiles=torch.zeros(n, dtype=torch.int32, device="cuda"),
                 depth=torch.zeros(n, dtype=torch.int32, device="cuda"),
                 stats=torch.zeros(msgs.MS_STATS_WORDS, dtype=torch.int32, device="cuda"))
        p = msgs.ms_proj_t(msgs._ptr(t["rec"]), msgs._ptr(t["rect"]), msgs._ptr(t["n_tiles"]),
                           msgs._ptr(t["depth"]), 0, 0, msgs._ptr(t["stats"]), n)
        return t, p

    m = msgs.MODES[mode]  # selective: views of one pose, the pruning launch
    joint = [proj() for _ in cams]
    msgs.ms_project_views(ds.struct, [msgs.camera_struct(c) for c in cams], m,
                          [p for _, p in joint])
    for (tj, _), cam in zip(joint, cams):
        ta, pa = proj()
        msgs.ms_project(ds.struct, msgs.camera_struct(cam), m, pa)
        torch.cuda.synchronize()
        assert int(ta["stats"][0]) > 65536  # survivors: more than one 16-bit count
        for k in ta:
            assert ta[k].equal(tj[k]), k
        del ta, pa


@pytest.mark.parametrize("n_views", [1, 4, 6])
def test_training_projection_updates_ranges_like_the_oracle(cuda, n_views):
    """Multi-scale training (Alg. 2): ms_project_views_update renders each
    view with the coverage ranges as they stand, then applies UpdateRange
    (Eq. 5) for the view's level.  Over three steps of views at the levels'
    creation scales (1x, 4x, 16x, 64x of orbit cameras, repeated for more
    than four views), every view's selection mask and coverage and the
    ranges after every step equal the oracle's sequence of footprints and
    or_update_range calls, bit for bit; a view with level 0 updates
    nothing."""
    sc = inputs.multiscale_scene(n=30_011, seed=5)       # fresh ranges (0, +inf)
    ds = msgs.DeviceScene(sc)
    ref = sc.copy()
    for step in range(3):
        orbit = inputs.orbit_cameras(n_views, seed=20 + step, radius=25.0, width=628,
                                     height=416)
        levels = [(v % 4) + 1 for v in range(n_views)]
        if n_views == 6:
            levels[5] = 0                                  # renders, updates nothing
        cams = [inputs.downscale(c, 4 ** (l - 1) if l else 2) for c, l in zip(orbit, levels)]
        rs = renderers(sc, cams)
        msgs.ms_project_views_update(ds.struct, [msgs.camera_struct(c) for c in cams],
                                     msgs.MODES["selective"], levels, [r.proj for r in rs])
        cuda.cuda.synchronize()
        for v, (cam, lv, r) in enumerate(zip(cams, levels, rs)):
            fp = oracle.footprints(ref, cam, "selective")
            got_mask = np.unpackbits(r.mask.cpu().numpy().view(np.uint8),
                                     bitorder="little")[:sc.n].astype(bool)
            np.testing.assert_array_equal(got_mask, fp["selected"] == 1, err_msg=f"view {v}")
            np.testing.assert_array_equal(r.cover.cpu().numpy()[:sc.n].view(np.uint32),
                                          fp["cover"].view(np.uint32))
            if lv:
                oracle.update_range(ref, cam, lv)
        np.testing.assert_array_equal(ds.s_max.cpu().numpy().view(np.uint32),
                                      np.ascontiguousarray(ref.s_max, np.float32).view(np.uint32))
        np.testing.assert_array_equal(ds.s_min.cpu().numpy().view(np.uint32),
                                      np.ascontiguousarray(ref.s_min, np.float32).view(np.uint32))
    assert np.isfinite(ref.s_max).sum() > 1000 and (ref.s_max > 0).sum() > 1000
