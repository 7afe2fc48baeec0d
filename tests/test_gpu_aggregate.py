"""ms_aggregate (AggregateGaussians, Alg. 1) through the C ABI against the
oracle on the same seeded scenes and cameras: the same voxels (bit-exact:
the small-Gaussian test and the voxel keys are FP32 decisions taken the
same way), in the same order, with the averaged attributes within FP32
summation error."""
import numpy as np
import pytest

import oracle
import paper_2311_17089_gb300 as msgs
from paper_2311_17089_gb300 import inputs

from gpu_util import require_cuda

pytestmark = pytest.mark.gpu
FIELDS = ("mean", "log_scale", "quat", "opacity", "color")


def _extent(cams):
    return float(max(np.abs(np.asarray(c.campos, np.float32)).max() for c in cams))


def _fine_scene(n, seed, sh_degree=3):
    """Level-1 Gaussians only (the input of the first aggregation); plain
    RGB colour for sh_degree -1."""
    sc = inputs.multiscale_scene(n=n, seed=seed, split=(1.0, 0.0, 0.0, 0.0), box=4.0,
                                 cluster_sigma=0.8, n_clusters=16, sh_degree=max(sh_degree, 0))
    sc.n_levels = 4
    if sh_degree < 0:
        sc.color = np.random.default_rng(seed).uniform(0, 1, (n, 3)).astype(np.float32)
        sc.sh_degree = -1
    return sc


def _compare(g, o):
    assert g["mean"].shape[0] == o["mean"].shape[0]
    np.testing.assert_allclose(g["mean"], o["mean"], rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(g["log_scale"], o["log_scale"], rtol=0, atol=2e-5)
    np.testing.assert_allclose(g["quat"], o["quat"], rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(g["opacity"], o["opacity"], rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(g["color"], o["color"], rtol=2e-5, atol=2e-6)


@pytest.mark.parametrize("level_m,deg", [(2, 3), (3, 1), (4, -1)])
def test_aggregate_level_matches_oracle(level_m, deg):
    require_cuda()
    sc = _fine_scene(30_000, seed=level_m, sh_degree=deg)
    base = inputs.orbit_cameras(6, seed=level_m, radius=10.0, width=512, height=384)
    cams = [inputs.downscale(c, 4 ** (level_m - 1)) for c in base]
    B = _extent(base)
    o, keys, smin = oracle.aggregate(sc, cams, level_m, B)
    assert len(keys) > 10
    ds = msgs.DeviceScene(sc)
    g = msgs.aggregate_level(ds, cams, level_m, B)
    gn = {k: g[k].cpu().numpy() for k in FIELDS}
    _compare(gn, o)
    assert (g["level"].cpu().numpy() == level_m).all()
    assert (g["s_max"].cpu().numpy() == 0).all() and np.isinf(g["s_min"].cpu().numpy()).all()


def test_aggregate_all_levels_in_sequence():
    """l_m = 2, 3, 4 in turn, each level appended before the next (the
    coarser levels aggregate the finer inserted ones too), on both sides."""
    require_cuda()
    sc = _fine_scene(20_000, seed=7, sh_degree=2)
    base = inputs.orbit_cameras(4, seed=7, radius=10.0, width=512, height=384)
    B = _extent(base)
    osc = sc.copy()
    gsc = sc.copy()
    for lm in (2, 3, 4):
        cams = [inputs.downscale(c, 4 ** (lm - 1)) for c in base]
        o, keys, _ = oracle.aggregate(osc, cams, lm, B)
        g = msgs.aggregate_level(msgs.DeviceScene(gsc), cams, lm, B)
        gn = {k: g[k].cpu().numpy() for k in FIELDS}
        _compare(gn, o)
        for s, new in ((osc, o), (gsc, gn)):
            m = len(new["mean"])
            s.mean = np.concatenate([s.mean, new["mean"]])
            s.log_scale = np.concatenate([s.log_scale, new["log_scale"]])
            s.quat = np.concatenate([s.quat, new["quat"]])
            s.opacity = np.concatenate([s.opacity, new["opacity"]])
            s.color = np.concatenate([s.color, new["color"]])
            s.level = np.concatenate([s.level, np.full(m, lm, np.uint8)])
            s.s_max = np.concatenate([s.s_max, np.zeros(m, np.float32)])
            s.s_min = np.concatenate([s.s_min, np.full(m, np.inf, np.float32)])
    assert gsc.n == osc.n > sc.n


def test_aggregate_capacity_and_empty():
    torch = require_cuda()
    sc = _fine_scene(5_000, seed=9, sh_degree=0)
    base = inputs.orbit_cameras(2, seed=9, radius=10.0, width=256, height=192)
    cams = [inputs.downscale(c, 4) for c in base]
    B = _extent(base)
    o, keys, _ = oracle.aggregate(sc, cams, 2, B)
    ds = msgs.DeviceScene(sc)
    # a capacity below the voxel count: the first `capacity` voxels, and the
    # count reported
    ws_b = msgs.ms_aggregate_workspace_bytes(sc.n)
    ws = torch.empty(ws_b, dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(2, dtype=torch.int64, device="cuda")
    cap = 3
    bufs = dict(mean=torch.zeros((cap, 3), device="cuda"), log_scale=torch.zeros((cap, 3), device="cuda"),
                quat=torch.zeros((cap, 4), device="cuda"), opacity=torch.zeros(cap, device="cuda"),
                color=torch.zeros((cap, 1, 3), device="cuda"),
                level=torch.zeros(cap, dtype=torch.uint8, device="cuda"),
                s_max=torch.zeros(cap, device="cuda"), s_min=torch.zeros(cap, device="cuda"))
    out = msgs.ms_scene_t(cap, 4, 0, *(msgs._ptr(bufs[k]) for k in
                                       ("mean", "log_scale", "quat", "opacity", "color", "level",
                                        "s_max", "s_min")), 0, 0)
    msgs.ms_aggregate(ds.struct, [msgs.camera_struct(c) for c in cams], 2, B, out, cap,
                      msgs._ptr(n_out), msgs._ptr(ws), ws_b)
    torch.cuda.synchronize()
    assert int(n_out[0]) == len(keys) > cap and int(n_out[1]) == 0
    np.testing.assert_allclose(bufs["mean"].cpu().numpy(), o["mean"][:cap], rtol=2e-6, atol=2e-6)
    # no camera: nothing is splatted, nothing is small
    g = msgs.aggregate_level(ds, [], 2, B)
    assert g["mean"].shape[0] == 0
