"""The render server (ms_serve_*): served frames match the oracle (sampled
tiles, 2e-4) and equal the same requests rendered alone through ms_project
-> ms_bin -> ms_raster, requests of one scene and mode share projection
passes, admission respects the memory budget and max_inflight, a request
that can never fit is refused, and a request whose duplicate capacity was
too small is re-rendered."""
import numpy as np
import pytest

import oracle
import paper_2311_17089_gb300 as msgs
from paper_2311_17089_gb300 import inputs

from gpu_util import assert_image_close, calibrated, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scenes():
    require_cuda()
    out = []
    for seed in (0, 1):
        sc = inputs.multiscale_scene(n=40_000, seed=seed, box=3.0, cluster_sigma=0.6,
                                     n_clusters=8)
        sc = calibrated(sc, inputs.orbit_cameras(4, seed=seed, radius=8.0, width=256,
                                                 height=192))
        out.append(sc)
    return out


def requests(k, seed):
    rng = np.random.default_rng(seed)
    base = inputs.orbit_cameras(k, seed=seed, radius=8.0, width=256, height=192)
    out = []
    for cam in base:
        s = int(rng.choice([1, 2, 4, 8, 16, 32]))
        out.append((int(rng.integers(0, 2)), inputs.downscale(cam, s),
                    ["selective", "all_levels"][int(rng.integers(0, 2))]))
    return out


def alone(ds, cam, mode):
    torch = require_cuda()
    r = msgs.Renderer(ds.n, cam.tiles_x * cam.tiles_y, 64 * ds.n, with_cover=False,
                      with_mask=False)
    img, _, _ = r.render(ds, cam, mode)
    r.check()
    torch.cuda.synchronize()
    return img.cpu().numpy()


def test_mixed_equals_alone(scenes):
    torch = require_cuda()
    dss = [msgs.DeviceScene(sc) for sc in scenes]
    reqs = requests(24, seed=3)
    with msgs.Server(max_gaussians=40_000, max_width=256, max_height=192,
                     mem_budget_bytes=2 << 30, max_inflight=8, n_streams=4) as srv:
        ids = [srv.add_scene(ds) for ds in dss]
        outs = [torch.empty((3, c.height, c.width), device="cuda") for _, c, _ in reqs]
        tickets = [srv.submit(ids[s], c, m, image_dev=o) for (s, c, m), o in zip(reqs, outs)]
        results = [srv.wait(t, 60.0) for t in tickets]
        st = srv.stats()
    assert all(r.status == msgs.MS_OK for r in results), [r.status for r in results]
    assert st.completed == len(reqs) and st.failed == 0
    assert 1 < st.peak_inflight <= 8
    assert st.proj_passes <= st.renders and st.proj_seconds > 0
    for (s, cam, mode), o, r in zip(reqs, outs, results):
        a = alone(dss[s], cam, mode)
        np.testing.assert_array_equal(o.cpu().numpy(), a)
        assert r.t_submit <= r.t_start <= r.t_done
    # served frames against the oracle: every third request, up to 12 sampled
    # tiles of each (all of a frame's tiles when it has fewer)
    rng = np.random.default_rng(11)
    for (s, cam, mode), o in list(zip(reqs, outs))[::3]:
        tiles = cam.tiles_x * cam.tiles_y
        pick = np.sort(rng.choice(tiles, min(tiles, 12), replace=False))
        want = oracle.render(scenes[s], cam, mode, tiles=pick)
        assert_image_close({"image": o.cpu().numpy()}, want, tiles=pick, cam=cam,
                           image_only=True)


def test_requests_of_one_scene_share_projection_passes(scenes):
    """Sixteen requests of one scene and mode queued at once are admitted in
    batches whose cameras share one ms_project_views pass; the frames are
    bit-identical to those rendered alone and to a server that projects
    every request by itself (max_batch_views = 1)."""
    torch = require_cuda()
    ds = msgs.DeviceScene(scenes[0])
    reqs = [(0, c, "selective") for _, c, _ in requests(16, seed=9)]
    got = {}
    for mb in (0, 1):
        with msgs.Server(max_gaussians=40_000, max_width=256, max_height=192,
                         mem_budget_bytes=2 << 30, max_inflight=16, n_streams=8,
                         max_batch_views=mb) as srv:
            sid = srv.add_scene(ds)
            outs = [torch.empty((3, c.height, c.width), device="cuda") for _, c, _ in reqs]
            tickets = [srv.submit(sid, c, m, image_dev=o) for (_, c, m), o in zip(reqs, outs)]
            results = [srv.wait(t, 60.0) for t in tickets]
            st = srv.stats()
        assert all(r.status == msgs.MS_OK for r in results)
        got[mb] = (outs, st)
    _, st_b = got[0]
    _, st_1 = got[1]
    assert st_1.proj_passes == st_1.renders
    assert st_b.proj_passes < st_b.renders, (st_b.proj_passes, st_b.renders)
    for (_, cam, mode), ob, o1 in zip(reqs, got[0][0], got[1][0]):
        a = alone(ds, cam, mode)
        np.testing.assert_array_equal(ob.cpu().numpy(), a)
        np.testing.assert_array_equal(o1.cpu().numpy(), a)


def test_request_that_can_never_fit_is_refused(scenes):
    """A request whose buffers exceed the whole arena finishes with
    MS_ERR_OOM; a small request fits a small arena and renders."""
    torch = require_cuda()
    ds = msgs.DeviceScene(scenes[0])
    big = inputs.orbit_cameras(1, seed=2, radius=8.0, width=256, height=192)[0]
    small = inputs.downscale(big, 32)
    with msgs.Server(max_gaussians=40_000, max_width=256, max_height=192,
                     mem_budget_bytes=8 << 20, max_inflight=2, n_streams=1,
                     initial_capacity=4_000_000) as srv:
        sid = srv.add_scene(ds)
        t_big = srv.submit(sid, big)
        r_big = srv.wait(t_big, 60.0)
    assert r_big.status == msgs.MS_ERR_OOM
    with msgs.Server(max_gaussians=40_000, max_width=256, max_height=192,
                     mem_budget_bytes=64 << 20, max_inflight=2, n_streams=1,
                     initial_capacity=40_000) as srv:
        sid = srv.add_scene(ds)
        out = torch.empty((3, small.height, small.width), device="cuda")
        r = srv.wait(srv.submit(sid, small, image_dev=out), 60.0)
    assert r.status == msgs.MS_OK
    np.testing.assert_array_equal(out.cpu().numpy(), alone(ds, small, "selective"))


def test_host_output_and_memory_admission(scenes):
    """A budget that holds about two requests: all still complete, the
    arena never exceeds the budget, images arrive in host memory."""
    torch = require_cuda()
    ds = msgs.DeviceScene(scenes[0])
    cam = inputs.downscale(inputs.orbit_cameras(1, seed=5, radius=8.0, width=256,
                                                height=192)[0], 1)
    cap = 400_000
    with msgs.Server(max_gaussians=40_000, max_width=256, max_height=192,
                     mem_budget_bytes=1 << 30, max_inflight=1, n_streams=1,
                     initial_capacity=cap) as probe:
        one = probe.wait(probe.submit(probe.add_scene(ds), cam), 60.0).bytes
    budget = int(2.5 * one)
    ref = alone(ds, cam, "selective")
    with msgs.Server(max_gaussians=40_000, max_width=256, max_height=192,
                     mem_budget_bytes=budget, max_inflight=16, n_streams=4,
                     initial_capacity=cap) as srv:
        sid = srv.add_scene(ds)
        hosts = [torch.empty((3, cam.height, cam.width)).pin_memory() for _ in range(10)]
        tickets = [srv.submit(sid, cam, "selective", image_host=h) for h in hosts]
        results = [srv.wait(t, 60.0) for t in tickets]
        st = srv.stats()
    assert all(r.status == msgs.MS_OK for r in results)
    assert st.arena_peak <= st.arena_bytes <= budget
    assert st.renders == st.completed + st.retries and st.issue_seconds > 0
    assert results[0].bytes == one
    assert st.peak_inflight * min(r.bytes for r in results) <= budget
    assert st.peak_inflight < len(hosts)
    for h in hosts:
        np.testing.assert_array_equal(h.numpy(), ref)


def test_capacity_overflow_is_retried(scenes):
    torch = require_cuda()
    ds = msgs.DeviceScene(scenes[1])
    reqs = [(0, c, m) for _, c, m in requests(6, seed=7)]
    with msgs.Server(max_gaussians=40_000, max_width=256, max_height=192,
                     mem_budget_bytes=1 << 30, max_inflight=4, n_streams=2,
                     initial_capacity=1024) as srv:
        sid = srv.add_scene(ds)
        outs = [torch.empty((3, c.height, c.width), device="cuda") for _, c, _ in reqs]
        tickets = [srv.submit(sid, c, m, image_dev=o) for (_, c, m), o in zip(reqs, outs)]
        results = [srv.wait(t, 60.0) for t in tickets]
    assert all(r.status == msgs.MS_OK for r in results)
    assert sum(r.retries for r in results) >= 1
    for (_, cam, mode), o, r in zip(reqs, outs, results):
        np.testing.assert_array_equal(o.cpu().numpy(), alone(ds, cam, mode))
        assert r.duplicates > 0


def test_poll_and_errors(scenes):
    ds = msgs.DeviceScene(scenes[0])
    cam = inputs.downscale(inputs.config2_camera(256, 192, distance=8.0), 4)
    with msgs.Server(max_gaussians=40_000, max_width=256, max_height=192,
                     mem_budget_bytes=1 << 30, max_inflight=2, n_streams=1) as srv:
        sid = srv.add_scene(ds)
        with pytest.raises(msgs.MsError):
            srv.submit(sid + 5, cam)                       # unknown scene
        with pytest.raises(msgs.MsError):
            srv.submit(sid, inputs.config2_camera(512, 192))  # larger than max_width
        t = srv.submit(sid, cam)
        r = srv.wait(t, 60.0)
        assert r.status == msgs.MS_OK
        with pytest.raises(msgs.MsError):
            srv.poll(t)                                    # a finished ticket is forgotten
        big = msgs.DeviceScene(inputs.single_level_scene(50_000, seed=1))
        with pytest.raises(msgs.MsError):
            srv.add_scene(big)                             # more than max_gaussians
