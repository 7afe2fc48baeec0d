"""ms_bin_noalloc: binning for callers that cannot allocate device memory.

Some callers own no device allocations of their own (an engine plugin whose
host application manages all device memory, a frame loop under a fixed
budget or a no-allocation rule), so they cannot hand ms_bin a workspace.
ms_bin_noalloc runs the same binning with the library's static scratch
array.  These tests call it through the C ABI and check, on consecutive
calls, that its tile lists, ranges and counts equal ms_bin's bit for bit
(the tolerance of every tile-list test), and that a frame rendered from its
lists is bit-identical to one rendered from ms_bin's.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import paper_2311_17089_gb300 as msgs
from paper_2311_17089_gb300 import inputs

pytestmark = pytest.mark.gpu


def _frame_bins(torch, r, ds, cam, mode):
    """ms_project then ms_bin with the caller's workspace; host copies."""
    cs = msgs.camera_struct(cam)
    msgs.ms_project(ds.struct, cs, msgs.MODES[mode], r.proj)
    msgs.ms_bin(r.proj, ds.n, cs, r.bins, msgs._ptr(r.ws), r.ws_bytes)
    rc, d, s = msgs.ms_bin_counts(r.bins)
    assert rc == msgs.MS_OK
    tiles = cam.tiles_x * cam.tiles_y
    return (d, s, r.gauss_idx[:d].clone(), r.ranges[:2 * tiles].clone())


def _noalloc_bins(torch, r, ds, cam, cap):
    """ms_bin_noalloc into separate output buffers; host copies."""
    dev = r.gauss_idx.device
    gidx = torch.full((cap,), -1, dtype=torch.int32, device=dev)
    ranges = torch.full((r.max_tiles * 2,), -1, dtype=torch.int32, device=dev)
    counts = torch.full((4,), -1, dtype=torch.int64, device=dev)
    bins = msgs.ms_bins_t(msgs._ptr(gidx), msgs._ptr(ranges), msgs._ptr(counts), cap)
    cs = msgs.camera_struct(cam)
    msgs.ms_bin_noalloc(r.proj, ds.n, cs, bins)
    rc, d, s = msgs.ms_bin_counts(bins)
    assert rc == msgs.MS_OK
    tiles = cam.tiles_x * cam.tiles_y
    return (d, s, gidx[:d].clone(), ranges[:2 * tiles].clone()), bins, (gidx, ranges, counts)


def test_noalloc_binning_equals_workspace_binning_on_consecutive_calls():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("needs a CUDA device")
    sc = inputs.multiscale_scene(n=60_000, seed=4)
    sc.s_max[:] = np.inf          # every level selected by its range
    sc.s_min[:] = 0.0
    ds = msgs.DeviceScene(sc)
    big = inputs.config2_camera()
    cams = [inputs.downscale(big, 4), inputs.downscale(big, 16), inputs.downscale(big, 4)]
    cap = 600_000
    r = msgs.Renderer(sc.n, big.tiles_x * big.tiles_y, cap)
    for cam in cams:                      # consecutive calls share the array
        want = _frame_bins(torch, r, ds, cam, "selective")
        got, bins, keep = _noalloc_bins(torch, r, ds, cam, cap)
        assert want[0] > 1000 and got[0] == want[0] and got[1] == want[1]
        assert torch.equal(got[2], want[2])
        assert torch.equal(got[3], want[3])
        # the same frame rendered from either set of lists
        img_a, _, _ = r.images(cam)
        img_b, _, _ = r.images(cam)
        cs = msgs.camera_struct(cam)
        msgs.ms_raster(r.proj, r.bins, cs, msgs._ptr(img_a), 0, 0, 0, msgs._ptr(r.rws),
                       r.rws_bytes)
        msgs.ms_raster(r.proj, bins, cs, msgs._ptr(img_b), 0, 0, 0, msgs._ptr(r.rws),
                       r.rws_bytes)
        torch.cuda.synchronize()
        # identical lists and records: the same kernel gives the same bits
        assert torch.equal(img_a, img_b)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("needs a CUDA device")
    cam = inputs.config2_camera()
    proj = msgs.ms_proj_t()
    proj.n = 2_000_000
    bins = msgs.ms_bins_t(0, 0, 0, 1 << 24)
    with pytest.raises(msgs.MsError) as e:
        msgs.ms_bin_noalloc(proj, 2_000_000, msgs.camera_struct(cam), bins)
    assert e.value.code == msgs.MS_ERR_INVALID_ARG
    assert "static" in str(e.value)
