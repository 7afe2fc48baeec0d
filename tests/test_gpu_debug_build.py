"""The debug build (libmsgs_debug.so, -DMS_DEBUG): its index checks stay
silent on a correct frame, which still matches the oracle, and report a
corrupted tile list as MS_ERR_BOUNDS through the status word instead of
trapping; the kernels clamp the access as the release build does.  Run in
a child process, since the binding picks its library at import."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import numpy as np
import torch
import oracle
import paper_2311_17089_gb300 as msgs
from paper_2311_17089_gb300 import inputs
from gpu_util import assert_image_close, gpu_frame

assert msgs.DEBUG and msgs.LIB_PATH.endswith("libmsgs_debug.so")
sc = inputs.multiscale_scene(n=4000, seed=0, split=(0.75, 0.25), box=1.0,
                             cluster_sigma=0.3, n_clusters=8)
sc = oracle.calibrate(sc, inputs.orbit_cameras(4, seed=1, radius=4.0, width=96, height=80))
cam = inputs.pinhole((0.0, 0.0, -4.0), (0, 0, 0), (0, -1, 0), 96, 80, 60.0)
o = oracle.render(sc, cam, "selective")
for strategy in ("tile", "list", "group16"):
    g = gpu_frame(sc, cam, "selective", strategy=strategy)   # asserts MS_OK
    assert_image_close(g, o)
# the sweep's path (pruned multi-view projection, shared sort split into
# per-frame orders, ordered binning) under the debug checks: silent, and the
# frames equal the frames rendered one by one
cams = [inputs.downscale(cam, s) for s in (1, 2, 4)]
ds0 = msgs.DeviceScene(sc)
for mode in ("selective", "all_levels"):
    alone = [msgs.Renderer(sc.n, c.tiles_x * c.tiles_y, 64 * sc.n) for c in cams]
    want = [r.render(ds0, c, mode) for r, c in zip(alone, cams)]
    rs = [msgs.Renderer(sc.n, c.tiles_x * c.tiles_y, 64 * sc.n, with_cover=False)
          for c in cams]
    order = msgs.DepthOrder(sc.n, split_views=len(cams))
    got = msgs.render_views(ds0, rs, cams, mode, order=order)
    for r in alone + rs:
        r.check()                                  # MS_OK, no index check fired
    torch.cuda.synchronize()
    for w, gimg in zip(want, got):
        for a, b in zip(w, gimg):
            assert a.equal(b)
# a tile list entry beyond the projection's Gaussians: each raster kernel
# clamps it and the debug checks report it
ds = msgs.DeviceScene(sc)
for strategy in ("tile", "list", "group16"):
    r = msgs.Renderer(sc.n, cam.tiles_x * cam.tiles_y, 64 * sc.n)
    r.render(ds, cam, "selective", strategy=strategy)
    d, _ = r.check()
    assert d > 0
    # the first entry of the longest list: every raster kernel stages it
    rg = r.ranges[:2 * cam.tiles_x * cam.tiles_y].view(-1, 2).long()
    t = int(torch.argmax(rg[:, 1] - rg[:, 0]))
    r.gauss_idx[int(rg[t, 0])] = sc.n + 7
    img, ft, nc = r.images(cam)
    msgs.ms_raster_ex(r.proj, r.bins, msgs.camera_struct(cam), msgs._ptr(img), 0, 0, 0,
                      msgs._ptr(r.rws), r.rws_bytes, msgs.STRATEGIES[strategy])
    try:
        msgs.ms_bin_counts(r.bins)
        raise AssertionError("the corrupted list was not reported")
    except msgs.MsError as e:
        assert e.code == msgs.MS_ERR_BOUNDS, e
    torch.cuda.synchronize()
print("debug build ok")
'''.replace("ROOT", repr(ROOT))


def test_debug_build_checks_are_silent_when_correct_and_report_corruption():
    env = dict(os.environ, MSGS_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug build ok" in r.stdout
