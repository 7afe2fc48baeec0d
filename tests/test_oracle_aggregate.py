"""Pins of the oracle's AggregateGaussians (Alg. 1; supplementary "Details of
Gaussian Aggregation Algorithm") against values the paper's definitions fix
by construction: the normalisation and voxel index at special points, the
grouping of Gaussians placed in known voxels, averages of constructed
members, the closed-form pixel coverage of isotropic Gaussians on the
optical axis, and the enlargement's stated goal (coverage S_T = 2 px)."""
import math

import numpy as np
import pytest

from paper_2311_17089_gb300 import inputs


def _scene(means, log_scales, opacities, levels, sh_degree=-1, seed=0):
    n = len(means)
    rng = np.random.default_rng(seed)
    color = (rng.uniform(0, 1, (n, 3)) if sh_degree < 0 else
             rng.normal(0, 0.3, (n, (sh_degree + 1) ** 2, 3))).astype(np.float32)
    quat = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    return inputs.Scene(np.asarray(means, np.float32),
                        np.repeat(np.asarray(log_scales, np.float32)[:, None], 3, 1),
                        quat, np.asarray(opacities, np.float32), color,
                        np.asarray(levels, np.uint8), 4, sh_degree,
                        np.zeros(n, np.float32), np.full(n, np.inf, np.float32))


def _axis_camera(z_cam, width=128, height=128):
    """Camera on the optical axis at (0, 0, z_cam) looking at +z."""
    return inputs.pinhole((0.0, 0.0, z_cam), (0.0, 0.0, z_cam + 1.0), (0.0, -1.0, 0.0),
                          width, height, 60.0)


def test_voxel_key_at_special_points(orc):
    """Per component: x / B inside [-B, B], sign(x) (2 - B/|x|) outside;
    floor(400 / l_m) voxels per axis over [-2, 2]."""
    B = 10.0
    for lm, R in ((2, 200), (3, 133), (4, 100)):
        def key(x, y, z):
            return orc.voxel_key([x, y, z], B, lm)
        # the origin maps to the middle voxel R/2 (t = 2 * R/4 exactly)
        c = R // 2
        assert key(0, 0, 0) == (c * R + c) * R + c
        # x = 2B normalises to 1.5 (outer region), -2B to -1.5: voxels
        # floor(3.5 R / 4) and floor(0.5 R / 4)
        assert key(2 * B, 0, 0) == (c * R + c) * R + math.floor(3.5 * R / 4)
        assert key(0, -2 * B, 0) == (c * R + math.floor(0.5 * R / 4)) * R + c
        # far away saturates at the last voxel, never beyond
        assert key(0, 0, 1e30) == ((R - 1) * R + c) * R + c
        assert key(0, 0, -1e30) == (0 * R + c) * R + c
        # on the cube face both branches give 1 (voxel floor(3R/4)), and just
        # inside / just outside stay within one voxel of it (continuity)
        face = (c * R + c) * R + math.floor(3 * R / 4)
        assert key(B, 0, 0) == face
        assert abs(key(B * (1 - 1e-6), 0, 0) - face) <= 1
        assert abs(key(B * (1 + 1e-6), 0, 0) - face) <= 1


def test_groups_averages_and_enlargement(orc):
    """Three small Gaussians in one voxel and two in another (on the optical
    axis of the only camera), a large one, a coarse-level one and one
    behind the camera: two new Gaussians with the members' averages and
    the log-scale raised by ln(S_T / S_avg), S being the closed-form
    coverage 2 sqrt(2 ln(255 sigma)) f e^s / z of an on-axis isotropic
    Gaussian."""
    z_cam = -10.0
    cam = _axis_camera(z_cam)
    B = 10.0
    vox = 4.0 / 200 * B          # l_m = 2: voxel edge in world units (0.2)
    za = 2.0 * vox + 0.5 * vox   # centre of the voxel at index 100 + 2 along z
    zb = 5.0 * vox + 0.5 * vox
    d = 0.1 * vox
    means = [(0, 0, za - d), (0, 0, za), (0, 0, za + d), (0, 0, zb - d), (0, 0, zb + d),
             (0, 0, za),          # large: not small
             (0, 0, zb),          # level 2: not an input of l_m = 2
             (0, 0, z_cam - 5)]   # behind the camera: never splatted
    ls = [-5.0, -4.8, -4.9, -5.2, -5.1, -1.0, -5.0, -5.0]
    op = [0.2, 0.4, 0.6, 0.5, 0.7, 0.5, 0.5, 0.5]
    lv = [1, 1, 1, 1, 1, 1, 2, 1]
    sc = _scene(means, ls, op, lv, sh_degree=1)
    new, keys, smin = orc.aggregate(sc, [cam], 2, B)
    assert len(keys) == 2 and keys[0] < keys[1]

    def cover(i):
        z = means[i][2] - z_cam
        return 2 * math.sqrt(2 * math.log(255 * op[i])) * cam.fx * math.exp(ls[i]) / z

    for i in range(5):
        assert smin[i] == pytest.approx(cover(i), rel=1e-5)
    assert smin[5] > 2.0
    assert np.isinf(smin[6]) and np.isinf(smin[7])
    for g, members in ((0, [0, 1, 2]), (1, [3, 4])):
        np.testing.assert_allclose(new["mean"][g], np.mean([means[i] for i in members], 0),
                                   rtol=1e-6, atol=1e-7)
        assert new["opacity"][g] == pytest.approx(np.mean([op[i] for i in members]), rel=1e-6)
        s_avg = np.mean([cover(i) for i in members])
        want = np.mean([ls[i] for i in members]) + math.log(2.0 / s_avg)
        np.testing.assert_allclose(new["log_scale"][g], want, rtol=0, atol=2e-5)
        np.testing.assert_allclose(new["color"][g], sc.color[members].mean(0), rtol=1e-6,
                                   atol=1e-7)
        np.testing.assert_allclose(new["quat"][g], [1, 0, 0, 0], atol=0)


def test_single_member_voxel_is_enlarged_to_the_threshold(orc):
    """The stated goal of the enlargement: the new Gaussian's pixel coverage
    is S_T = 2 px (exact for one isotropic member, S being proportional to
    the scale)."""
    cam = _axis_camera(-10.0)
    sc = _scene([(0, 0, 0.05)], [-4.5], [0.6], [1])
    new, keys, smin = orc.aggregate(sc, [cam], 2, 10.0)
    assert len(keys) == 1 and smin[0] < 2.0
    out = _scene(new["mean"], new["log_scale"][:, 0], new["opacity"], [2])
    cov, *_ = orc.coverage64(out, cam)
    assert cov[0] == pytest.approx(2.0, rel=1e-5)


def test_smallest_coverage_over_cameras_decides(orc):
    """A Gaussian large in a near camera but small in a far one is small
    (its minimal coverage over the cameras counts); one large in both is
    not."""
    near, far = _axis_camera(-2.0), _axis_camera(-40.0)
    sc = _scene([(0, 0, 0.0), (0, 0, 0.5)], [-3.0, 0.0], [0.5, 0.5], [1, 1])
    _, keys, smin = orc.aggregate(sc, [near], 2, 10.0)
    assert len(keys) == 0 and (smin > 2.0).all()
    _, keys, smin = orc.aggregate(sc, [near, far], 2, 10.0)
    assert len(keys) == 1 and smin[0] < 2.0 < smin[1]
