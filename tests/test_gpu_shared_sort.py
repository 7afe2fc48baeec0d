"""One depth sort for the frames of one pose (a camera at several
resolutions, as in a multi-scale sweep): ms_project_views_union writes the
union of the Gaussians the views list, ms_sort_depth orders it by (depth
bits, index) and every frame's ms_bin_ordered must then give exactly the
tile lists, ranges and counts ms_bin gives that frame with its own sort,
and exactly the same images."""
import numpy as np
import pytest

import paper_2311_17089_gb300 as msgs
from paper_2311_17089_gb300 import inputs

from gpu_util import calibrated, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    return require_cuda()


@pytest.fixture(scope="module")
def ms_scene_50k():
    sc = inputs.multiscale_scene(n=50_000, seed=0)
    return calibrated(sc, inputs.orbit_cameras(8, seed=1, radius=25.0))


def degenerate_scene():
    """A ragged count with invalid Gaussians of every kind."""
    sc = inputs.single_level_scene(n=3001, seed=6)
    sc.quat[0:10] = 0.0
    sc.mean[10:20, 0] = np.nan
    sc.log_scale[20:30] = -30.0
    sc.log_scale[30:35] = 30.0
    sc.opacity[35:45] = 1.0 / 255.0
    sc.mean[50:60, 2] = -3.0
    return sc


def sweep_cams(scales=inputs.SCALES):
    return [inputs.downscale(inputs.config2_camera(), s) for s in scales]


def renderers(n, cams, cover=True):
    # without coverage output, selective views of one pose take the
    # projection launch that leaves out footprints ruled out by the bound
    return [msgs.Renderer(n, c.tiles_x * c.tiles_y, 16 * n + 4096, with_cover=cover)
            for c in cams]


def bins_of(torch, r):
    counts = r.counts.cpu().numpy()
    d = int(counts[0])
    return (r.gauss_idx[:d].cpu().numpy(), r.ranges.cpu().numpy().copy(), counts.copy())


def run_both(torch, sc, cams, mode, views=None, cover=True, split=False):
    ds = msgs.DeviceScene(sc)
    own, shared = renderers(sc.n, cams), renderers(sc.n, cams, cover)
    order = msgs.DepthOrder(sc.n, split_views=len(cams) if split else 0)
    out_own = msgs.render_views(ds, own, cams, mode)
    out_shared = msgs.render_views(ds, shared, cams, mode, order=order, order_views=views)
    torch.cuda.synchronize()
    return ds, own, shared, order, out_own, out_shared


def expected_order(own, n, views=None):
    """The union's indices sorted by (depth key as uint32, index), from the
    per-frame projections (the union's frames share the depth keys)."""
    views = range(len(own)) if views is None else sorted(views)
    listed = np.zeros(n, dtype=bool)
    for v in views:
        listed |= own[v].n_tiles[:n].cpu().numpy() > 0
    # (the union's flags hold, per Gaussian, the mask of the views listing it)
    depth = own[views[0]].depth[:n].cpu().numpy().view(np.uint32)
    idx = np.nonzero(listed)[0]
    return idx[np.argsort(depth[idx], kind="stable")], listed


@pytest.mark.parametrize("mode,cover", [("selective", True), ("selective", False),
                                        ("all_levels", True)])
def test_shared_order_bins_like_own_sort(cuda, ms_scene_50k, mode, cover):
    torch = cuda
    cams = sweep_cams()
    sc = ms_scene_50k
    _, own, shared, order, out_own, out_shared = run_both(torch, sc, cams, mode, cover=cover)
    want, listed = expected_order(own, sc.n)
    stats = order.stats.cpu().numpy()
    assert int(stats[0]) == len(want)
    assert np.array_equal(order.flags[:sc.n].cpu().numpy() > 0, listed)
    mask = np.zeros(sc.n, dtype=np.int64)
    for v, r in enumerate(own):
        mask |= (r.n_tiles[:sc.n].cpu().numpy() > 0).astype(np.int64) << v
    assert np.array_equal(order.flags[:sc.n].cpu().numpy().astype(np.int64), mask)
    assert np.array_equal(order.order[:len(want)].cpu().numpy(), want.astype(np.int32))
    # the union is larger than the finest frame's list (coarse levels are
    # listed in the coarse frames only), so the skipping path is exercised
    assert len(want) > int(own[0].stats[0].item())
    for v, (a, b) in enumerate(zip(own, shared)):
        ia, ra, ca = bins_of(torch, a)
        ib, rb, cb = bins_of(torch, b)
        assert np.array_equal(ca, cb), v
        assert np.array_equal(ra, rb), v
        assert np.array_equal(ia, ib), v
    for v, (x, y) in enumerate(zip(out_own, out_shared)):
        for k in range(3):
            assert x[k].equal(y[k]), (v, k)


@pytest.mark.parametrize("mode", ["selective", "all_levels"])
def test_split_order_bins_like_own_sort(cuda, ms_scene_50k, mode):
    """ms_split_order gives every frame its own part of the shared order:
    exactly the frame's listed Gaussians in (depth bits, index) order, its
    count in the view stats, and lists, ranges, counts and images equal to
    ms_bin's."""
    torch = cuda
    cams = sweep_cams()
    sc = ms_scene_50k
    _, own, shared, order, out_own, out_shared = run_both(torch, sc, cams, mode, cover=False,
                                                          split=True)
    depth = own[0].depth[:sc.n].cpu().numpy().view(np.uint32)
    for v, r in enumerate(own):
        idx = np.nonzero(r.n_tiles[:sc.n].cpu().numpy() > 0)[0]
        want = idx[np.argsort(depth[idx], kind="stable")]
        st = order.view_stats[v].cpu().numpy()
        assert int(st[0]) == len(want), v
        assert int(st[4]) == 0 and int(st[5]) == 0, v
        assert np.array_equal(order.view_orders[v][:len(want)].cpu().numpy(),
                              want.astype(np.int32)), v
    for v, (a, b) in enumerate(zip(own, shared)):
        for x, y in zip(bins_of(torch, a), bins_of(torch, b)):
            assert np.array_equal(x, y), v
    for v, (x, y) in enumerate(zip(out_own, out_shared)):
        for k in range(3):
            assert x[k].equal(y[k]), (v, k)


def test_split_order_ragged_and_subsets(cuda):
    """A ragged scene with invalid Gaussians, the union over some of the
    views (the others sort their own lists), and an empty view."""
    torch = cuda
    sc = degenerate_scene()
    cams = [inputs.downscale(inputs.config1_camera(), s) for s in (1, 2, 4, 8)]
    for views in (None, (1, 3)):
        _, own, shared, order, out_own, out_shared = run_both(torch, sc, cams, "selective",
                                                              views, split=True)
        for a, b in zip(own, shared):
            for x, y in zip(bins_of(torch, a), bins_of(torch, b)):
                assert np.array_equal(x, y)
        for x, y in zip(out_own, out_shared):
            for k in range(3):
                assert x[k].equal(y[k])


def test_shared_order_ragged_invalid_scene(cuda):
    torch = cuda
    sc = degenerate_scene()
    cams = [inputs.downscale(inputs.config1_camera(), s) for s in (1, 2, 4, 8)]
    _, own, shared, order, out_own, out_shared = run_both(torch, sc, cams, "selective")
    want, _ = expected_order(own, sc.n)
    assert int(order.stats[0].item()) == len(want)
    assert np.array_equal(order.order[:len(want)].cpu().numpy(), want.astype(np.int32))
    for a, b in zip(own, shared):
        for x, y in zip(bins_of(torch, a), bins_of(torch, b)):
            assert np.array_equal(x, y)
    for x, y in zip(out_own, out_shared):
        for k in range(3):
            assert x[k].equal(y[k])


def test_single_view_union(cuda, ms_scene_50k):
    """One view: the union is that view's list and the order its own."""
    torch = cuda
    cams = sweep_cams((2,))
    sc = ms_scene_50k
    _, own, shared, order, out_own, out_shared = run_both(torch, sc, cams, "selective")
    assert int(order.stats[0].item()) == int(own[0].stats[0].item())
    for x, y in zip(bins_of(torch, own[0]), bins_of(torch, shared[0])):
        assert np.array_equal(x, y)
    for k in range(3):
        assert out_own[0][k].equal(out_shared[0][k])


@pytest.mark.parametrize("views", [(0, 1, 2), (2, 5), (7,)])
def test_union_of_some_views(cuda, ms_scene_50k, views):
    """The fine frames share a sort, the others sort their own lists."""
    torch = cuda
    cams = sweep_cams()
    sc = ms_scene_50k
    _, own, shared, order, out_own, out_shared = run_both(torch, sc, cams, "selective", views,
                                                          cover=False)
    want, _ = expected_order(own, sc.n, views)
    assert int(order.stats[0].item()) == len(want)
    assert np.array_equal(order.order[:len(want)].cpu().numpy(), want.astype(np.int32))
    for a, b in zip(own, shared):
        for x, y in zip(bins_of(torch, a), bins_of(torch, b)):
            assert np.array_equal(x, y)
    for x, y in zip(out_own, out_shared):
        for k in range(3):
            assert x[k].equal(y[k])


def test_views_outside_the_union_may_have_other_poses(cuda, ms_scene_50k):
    torch = cuda
    sc = ms_scene_50k
    a, b = inputs.orbit_cameras(2, seed=4, radius=25.0, width=400, height=300)
    cams = [a, inputs.downscale(a, 2), b]
    _, own, shared, order, out_own, out_shared = run_both(torch, sc, cams, "selective", (0, 1))
    for x, y in zip(out_own, out_shared):
        for k in range(3):
            assert x[k].equal(y[k])


def test_union_needs_one_pose(cuda, ms_scene_50k):
    sc = ms_scene_50k
    ds = msgs.DeviceScene(sc)
    a, b = inputs.orbit_cameras(2, seed=4, radius=25.0, width=400, height=300)
    rs = renderers(sc.n, [a, b])
    order = msgs.DepthOrder(sc.n)
    with pytest.raises(msgs.MsError) as e:
        order.project(ds, rs, [a, b])
    assert e.value.code == msgs.MS_ERR_INVALID_ARG
    css = [msgs.camera_struct(c) for c in (a, a)]
    for mask in (0, 4, 1 << 31):
        with pytest.raises(msgs.MsError) as e:
            msgs.ms_project_views_union(ds.struct, css, msgs.MODES["selective"],
                                        [r.proj for r in rs], mask, msgs._ptr(order.flags),
                                        msgs._ptr(order.stats))
        assert e.value.code == msgs.MS_ERR_INVALID_ARG


def test_ordered_binning_reports_capacity(cuda, ms_scene_50k):
    """A frame whose duplicates exceed its capacity reports it exactly as
    ms_bin does."""
    torch = cuda
    sc = ms_scene_50k
    cams = sweep_cams((1, 2))
    ds = msgs.DeviceScene(sc)
    rs = [msgs.Renderer(sc.n, c.tiles_x * c.tiles_y, 1024) for c in cams]
    order = msgs.DepthOrder(sc.n)
    msgs.render_views(ds, rs, cams, "selective", order=order)
    torch.cuda.synchronize()
    for r in rs:
        with pytest.raises(msgs.MsError) as e:
            r.check()
        assert e.value.code == msgs.MS_ERR_CAPACITY
