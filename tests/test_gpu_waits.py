"""Bounded device waits: the binning's decoupled look-backs give up after a
limit, report MS_ERR_TIMEOUT through ms_bin_counts and leave the context
usable, with no hang and no fault.  The limit is lowered for ms_bin only
(ms_debug_set_spin_limit, a test hook), so that predecessors that have not
published yet make a wait run out; every write on that path is guarded to
stay inside its buffer."""
import numpy as np
import pytest

import oracle
import paper_2311_17089_gb300 as msgs
from paper_2311_17089_gb300 import inputs

from gpu_util import assert_lists_equal, require_cuda

pytestmark = pytest.mark.gpu


def test_binning_wait_gives_up_and_context_stays_usable():
    torch = require_cuda()
    sc = inputs.multiscale_scene(n=120_000, seed=8)
    cam = inputs.downscale(inputs.config2_camera(), 2)
    cs = msgs.camera_struct(cam)
    ds = msgs.DeviceScene(sc)
    fp = oracle.footprints(sc, cam, "all_levels")
    off, idx = oracle.tile_lists(fp, cam)
    r = msgs.Renderer(sc.n, cam.tiles_x * cam.tiles_y, len(idx) + 4096)
    msgs.ms_project(ds.struct, cs, msgs.MODES["all_levels"], r.proj)
    codes = []
    try:
        msgs.ms_debug_set_spin_limit(1)
        for _ in range(6):
            msgs.ms_bin(r.proj, sc.n, cs, r.bins, msgs._ptr(r.ws), r.ws_bytes)
            try:
                rc, d, _ = msgs.ms_bin_counts(r.bins)
                codes.append(rc)
            except msgs.MsError as e:
                codes.append(e.code)
            if codes[-1] == msgs.MS_ERR_TIMEOUT:
                break
    finally:
        msgs.ms_debug_set_spin_limit(0)
    assert codes[-1] == msgs.MS_ERR_TIMEOUT, codes
    assert all(c in (msgs.MS_OK, msgs.MS_ERR_TIMEOUT) for c in codes), codes
    # the same binning with the default limit: exact again
    msgs.ms_bin(r.proj, sc.n, cs, r.bins, msgs._ptr(r.ws), r.ws_bytes)
    rc, d, surv = msgs.ms_bin_counts(r.bins)
    assert rc == msgs.MS_OK
    torch.cuda.synchronize()
    g = dict(D=d, gauss_idx=r.gauss_idx.cpu().numpy().view(np.uint32)[:d],
             ranges=r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)[:cam.tiles_x * cam.tiles_y])
    assert_lists_equal(g, off, idx)


def test_shared_sort_wait_gives_up_and_every_frame_reports_it():
    """The shared depth sort and its split (ms_sort_depth, ms_split_order)
    record a wait that gave up in the union's status, which every frame
    binned from the split order reports; with the default limit the
    frames' lists are exact again."""
    torch = require_cuda()
    sc = inputs.multiscale_scene(n=120_000, seed=8)
    cams = [inputs.downscale(inputs.config2_camera(), s) for s in (1, 2, 4)]
    ds = msgs.DeviceScene(sc)
    rs = [msgs.Renderer(sc.n, c.tiles_x * c.tiles_y, 64 * sc.n, with_cover=False)
          for c in cams]
    order = msgs.DepthOrder(sc.n, split_views=len(cams))

    def sweep():
        order.project(ds, rs, cams, "all_levels")
        order.sort()
        codes = []
        for k, (r, c) in enumerate(zip(rs, cams)):
            o, st = order.view_order(k)
            msgs.ms_bin_ordered(r.proj, sc.n, msgs.camera_struct(c), r.bins, o, st,
                                msgs._ptr(r.ws), r.ws_bytes)
            try:
                codes.append(msgs.ms_bin_counts(r.bins)[0])
            except msgs.MsError as e:
                codes.append(e.code)
        return codes

    seen = []
    try:
        msgs.ms_debug_set_spin_limit(1)
        for _ in range(6):
            seen.append(sweep())
            if msgs.MS_ERR_TIMEOUT in seen[-1]:
                break
    finally:
        msgs.ms_debug_set_spin_limit(0)
    assert msgs.MS_ERR_TIMEOUT in seen[-1], seen
    assert all(c in (msgs.MS_OK, msgs.MS_ERR_TIMEOUT) for s in seen for c in s), seen
    assert sweep() == [msgs.MS_OK] * len(cams)
    torch.cuda.synchronize()
    for r, c in zip(rs, cams):
        fp = oracle.footprints(sc, c, "all_levels")
        off, idx = oracle.tile_lists(fp, c)
        d = int(r.counts[0].item())
        g = dict(D=d, gauss_idx=r.gauss_idx.cpu().numpy().view(np.uint32)[:d],
                 ranges=r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)[:c.tiles_x * c.tiles_y])
        assert_lists_equal(g, off, idx)
