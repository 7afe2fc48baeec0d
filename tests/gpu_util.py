"""Shared helpers of the GPU parity tests: run the CUDA path through the
C-ABI binding and compare with the oracle on the same seeded inputs."""
import os

import numpy as np

import oracle
import paper_2311_17089_gb300 as msgs
from paper_2311_17089_gb300 import inputs

IMAGE_ATOL = 2e-4      # max abs per colour channel (FP32 path vs FP64 oracle)


def require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU parity tests need a CUDA device")
    return torch


def calibrated(scene, cams):
    """Coverage ranges written by the oracle (never by the CUDA path)."""
    return oracle.calibrate(scene.copy(), cams)


def gpu_frame(scene, cam, mode="selective", cap=None, ds=None, strategy="auto"):
    """Run ms_project -> ms_bin -> ms_raster_ex2(strategy); return host
    copies.  A strategy "tile@K" is the tile kernel on at most K CTAs per SM."""
    torch = require_cuda()
    ds = ds or msgs.DeviceScene(scene)
    cap = cap or max(4096, 16 * scene.n)
    strategy, _, ctas = strategy.partition("@")
    ctas = int(ctas) if ctas else 0
    r = msgs.Renderer(scene.n, cam.tiles_x * cam.tiles_y, cap)
    ne = torch.empty((cam.height, cam.width), dtype=torch.int32, device=ds.mean.device)
    img, ft, nc = r.render(ds, cam, mode, strategy=strategy, n_eval=ne, max_ctas_per_sm=ctas)
    rc, d, surv = msgs.ms_bin_counts(r.bins)
    if rc == msgs.MS_ERR_CAPACITY:
        r = msgs.Renderer(scene.n, cam.tiles_x * cam.tiles_y, max(d, 1))
        img, ft, nc = r.render(ds, cam, mode, strategy=strategy, n_eval=ne,
                               max_ctas_per_sm=ctas)
        rc, d, surv = msgs.ms_bin_counts(r.bins)
    assert rc == msgs.MS_OK, rc
    torch.cuda.synchronize()
    n = max(scene.n, 1)
    rec = r.rec.cpu().numpy().reshape(n, 12)
    out = dict(
        image=img.cpu().numpy(), final_t=ft.cpu().numpy(),
        n_contrib=nc.cpu().numpy().view(np.uint32),
        n_eval=ne.cpu().numpy().view(np.uint32),
        n_tiles=r.n_tiles.cpu().numpy().view(np.uint32)[:scene.n],
        depth=r.depth.cpu().numpy().view(np.uint32)[:scene.n],
        rect=r.rect.cpu().numpy().view(np.uint32).reshape(n, 2)[:scene.n],
        cover=r.cover.cpu().numpy()[:scene.n],
        mask=r.mask.cpu().numpy().view(np.uint32),
        rec=rec[:scene.n], D=d, survivors=surv,
        gauss_idx=r.gauss_idx.cpu().numpy().view(np.uint32)[:d],
        ranges=r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)[:cam.tiles_x * cam.tiles_y],
    )
    return out


def mask_bits(mask_words, n):
    bits = np.unpackbits(mask_words.view(np.uint8), bitorder="little")
    return bits[:n].astype(bool)


def assert_footprints_equal(g, fp, scene, cam):
    """K1 outputs bit-exact against the oracle's FP32 footprint."""
    n = scene.n
    listed = (fp["selected"] == 1) & (fp["ntiles"] > 0)
    np.testing.assert_array_equal(g["n_tiles"], np.where(listed, fp["ntiles"], 0))
    np.testing.assert_array_equal(g["cover"].view(np.uint32), fp["cover"].view(np.uint32))
    np.testing.assert_array_equal(mask_bits(g["mask"], n), fp["selected"] == 1)
    li = np.nonzero(listed)[0]
    np.testing.assert_array_equal(g["depth"][li], fp["depth"][li])
    r = fp["rect"][li].astype(np.uint32)
    np.testing.assert_array_equal(g["rect"][li, 0], r[:, 0] | (r[:, 1] << 16))
    np.testing.assert_array_equal(g["rect"][li, 1], r[:, 2] | (r[:, 3] << 16))
    rec = g["rec"][li]
    # the record holds the conic times -log2(e)/2 (a, c) and -log2(e) (b),
    # each one FP32 product
    kA = np.float32(-0.72134752044448170)
    kB = np.float32(-1.4426950408889634)
    con = fp["conic"][li].astype(np.float32)
    for col, want in ((0, fp["ux"][li]), (1, fp["uy"][li]), (2, kA * con[:, 0]),
                      (3, kB * con[:, 1]), (4, kA * con[:, 2]),
                      (5, scene.opacity[li])):
        np.testing.assert_array_equal(rec[:, col].view(np.uint32),
                                      np.ascontiguousarray(want, np.float32).view(np.uint32))
    rgb = oracle.colors(scene, cam)[li]
    np.testing.assert_allclose(rec[:, [6, 7, 8]], rgb, rtol=0, atol=2e-6)
    # the level-set half extents (ex, ey) in the record span the tile rectangle
    ux, uy, ex, ey = (rec[:, k].astype(np.float32) for k in (0, 1, 10, 11))
    q = np.float32(0.0625)
    x0 = np.maximum(np.floor((ux - ex) * q), 0).astype(np.int64)
    x1 = np.minimum(np.floor((ux + ex) * q), cam.tiles_x - 1).astype(np.int64)
    y0 = np.maximum(np.floor((uy - ey) * q), 0).astype(np.int64)
    y1 = np.minimum(np.floor((uy + ey) * q), cam.tiles_y - 1).astype(np.int64)
    np.testing.assert_array_equal(np.stack([x0, y0, x1, y1], 1), fp["rect"][li])
    return li


def assert_lists_equal(g, offsets, idx):
    D = len(idx)
    assert g["D"] == D
    np.testing.assert_array_equal(g["gauss_idx"], idx)
    counts = np.diff(offsets)
    got = g["ranges"][:, 1].astype(np.int64) - g["ranges"][:, 0]
    np.testing.assert_array_equal(got, counts)
    ne = counts > 0
    np.testing.assert_array_equal(g["ranges"][ne, 0], offsets[:-1][ne])


FLAG_LOG = []   # (test case, pixels compared, flagged pixels) of every image check


def _matches_alternative(alts, col, t, nc, ne, atol):
    """True when the GPU's pixel equals one of the oracle's alternatives:
    colour and T within atol, contributor and evaluation counts exact."""
    if alts is None:
        return False
    for row in alts:
        if (np.all(np.abs(col - row[:3]) <= atol) and abs(t - row[3]) <= atol
                and int(nc) == int(row[4]) and int(ne) == int(row[5])):
            return True
    return False


def assert_image_close(g, o, tiles=None, cam=None, atol=IMAGE_ATOL, label=None,
                       image_only=False):
    """Every pixel of the region against the oracle.  Where no decision sat
    within single-precision reach of a threshold (flag bit 0: alpha near
    1/255; bit 1: T (1 - alpha) near 1e-4), colour and final T must be within
    atol and the contributor and evaluation counts exact.  A flagged pixel
    may correctly take either branch of each flagged decision (a flip moves
    it by up to alpha T, beyond atol), so it must equal, to the same
    tolerance, one of the results the oracle reaches by taking those
    decisions each way (oracle.pixel_alternatives).  With image_only, g
    holds only the image (a served frame): colour alone is compared.
    Returns (max colour error on unflagged pixels, number of flagged
    pixels)."""
    flags = o["flags"]
    region = np.ones_like(flags, bool)
    if tiles is not None:
        region[:] = False
        for t in tiles:
            tx, ty = t % cam.tiles_x, t // cam.tiles_x
            region[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16] = True
    ok = region & (flags == 0)
    err = np.abs(g["image"] - o["image"])[:, ok]
    assert err.size == 0 or err.max() <= atol, err.max()
    if not image_only:
        terr = np.abs(g["final_t"] - o["final_t"])[ok]
        assert terr.size == 0 or terr.max() <= atol, terr.max()
        np.testing.assert_array_equal(g["n_contrib"][ok], o["n_contrib"][ok])
        # the evaluation count behind the benchmark's roofline (P_eval)
        np.testing.assert_array_equal(g["n_eval"][ok].astype(np.int64), o["n_eval"][ok])
    flagged = np.argwhere(region & (flags != 0))
    bad = []
    for y, x in flagged:
        alts = oracle.pixel_alternatives(o, int(x), int(y))
        if image_only:
            hit = alts is not None and any(
                np.all(np.abs(g["image"][:, y, x] - row[:3]) <= atol) for row in alts)
        else:
            hit = _matches_alternative(alts, g["image"][:, y, x], g["final_t"][y, x],
                                       g["n_contrib"][y, x], g["n_eval"][y, x], atol)
        if not hit:
            bad.append((int(x), int(y), None if alts is None else len(alts)))
    assert not bad, f"flagged pixels matching no alternative: {bad[:8]} ({len(bad)})"
    case = label or os.environ.get("PYTEST_CURRENT_TEST", "image").split(" ")[0]
    FLAG_LOG.append((case, int(region.sum()), len(flagged)))
    return float(err.max()) if err.size else 0.0, len(flagged)
