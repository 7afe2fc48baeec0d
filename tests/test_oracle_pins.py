"""Pins of the CPU oracle against facts that do not come from the oracle:
the paper's printed values, closed forms, brute force and library routines.

Each test is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand, a half width for a full width)
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2311_17089_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def one_gaussian(pos, log_scale, quat=(1, 0, 0, 0), opacity=0.9, rgb=(1, 1, 1),
                 level=1, n_levels=1):
    n = len(pos)
    pos = np.asarray(pos, np.float32).reshape(n, 3)
    ls = np.broadcast_to(np.asarray(log_scale, np.float32), (n, 3)).copy()
    q = np.broadcast_to(np.asarray(quat, np.float32), (n, 4)).copy()
    op = np.broadcast_to(np.asarray(opacity, np.float32), (n,)).copy()
    col = np.broadcast_to(np.asarray(rgb, np.float32), (n, 3)).copy()
    lv = np.broadcast_to(np.asarray(level, np.uint8), (n,)).copy()
    return inputs.Scene(pos, ls, q, op, col, lv, n_levels, -1,
                        np.zeros(n, np.float32), np.full(n, np.inf, np.float32))


# ---------------------------------------------------------------- constants

def test_golden_constants_match_oracle_thresholds(orc):
    """The thresholds the oracle applies are the paper's (Eq. 5, Eq. 6,
    Sec. 4.1): checked through behaviour at the boundaries, not by reading
    the source."""
    g = golden_constants()
    assert g["sigma_T"] == pytest.approx(1 / 255)
    cam = inputs.config1_camera()
    # a Gaussian whose coverage S we measure, then ranges around it
    sc = one_gaussian([[0, 0, 0]], [-3.0, -3.2, -2.9], level=2, n_levels=3)
    S = float(orc.footprints(sc, cam, "all_levels")["cover"][0])
    assert 2.0 < S < 20.0

    def sel(smax, smin, level=2, n_levels=3):
        s = sc.copy()
        s.level[:] = level
        s.n_levels = n_levels
        s.s_max[:] = smax
        s.s_min[:] = smin
        return int(orc.footprints(s, cam, "selective")["selected"][0])

    rmax, rmin = g["S_rel_max"], g["S_rel_min"]
    assert sel(S / (rmax * 0.999), 0.0) == 1      # S/S_max just under 1.5
    assert sel(S / (rmax * 1.001), 0.0) == 0      # just over 1.5
    # too small relative to S_min, but S >= S_T keeps it (S > 2 here)
    assert sel(S, S / (rmin * 0.9)) == 1
    # shrink the Gaussian below S_T: now the relative clause decides
    s2 = sc.copy()
    s2.log_scale[:] -= np.float32(math.log(S / 1.0))   # S -> ~1 px
    S2 = float(orc.footprints(s2, cam, "all_levels")["cover"][0])
    assert S2 < g["S_T"]
    for smin, want in [(S2 / (rmin * 1.001), 1), (S2 / (rmin * 0.999), 0)]:
        s3 = s2.copy()
        s3.level[:] = 2
        s3.n_levels = 3
        s3.s_min[:] = smin
        s3.s_max[:] = S2          # first clause passes (ratio 1)
        assert int(orc.footprints(s3, cam, "selective")["selected"][0]) == want
    # level exemptions (Sec. 4.1, last paragraph): finest level ignores the
    # upper bound, coarsest ignores the lower bound
    assert sel(S / 10.0, 0.0, level=1) == 1
    assert sel(S / 10.0, 0.0, level=3) == 0
    s4 = s2.copy()
    s4.level[:] = 3
    s4.n_levels = 3
    s4.s_max[:] = S2
    s4.s_min[:] = S2 * 100
    assert int(orc.footprints(s4, cam, "selective")["selected"][0]) == 1
    s4.level[:] = 2
    assert int(orc.footprints(s4, cam, "selective")["selected"][0]) == 0


# ---------------------------------------------------------------- coverage

def test_coverage_matches_supplementary_level_set_solution(orc):
    """Supplementary, 1-D analysis: e^{-a (S/2)^2} = 1/N gives
    S = 2 sqrt(ln N / a), a = 1/(2 s^2), N = 255, for a unit-opacity
    Gaussian.  An axis-aligned Gaussian on the optical axis has pixel std
    s = f e^{log_scale} / z along each image axis; coverage takes the
    narrower axis."""
    cam = inputs.config1_camera()
    z = 3.0
    for ls in ([-3.0, -2.5, -2.0], [-2.2, -3.1, -1.0], [-4.0, -4.0, -4.0]):
        sc = one_gaussian([[0, 0, 0]], ls, opacity=1.0)
        ls = [float(v) for v in sc.log_scale[0]]      # the stored FP32 values
        s_px = cam.fx * math.exp(min(ls[0], ls[1])) / z
        a = 1.0 / (2.0 * s_px ** 2)
        S_paper = 2.0 * math.sqrt(math.log(255.0) / a)
        cover64 = orc.coverage64(sc, cam)[0][0]
        assert cover64 == pytest.approx(S_paper, rel=1e-9)
        fp = orc.footprints(sc, cam, "all_levels")
        assert float(fp["cover"][0]) == pytest.approx(S_paper, rel=2e-6)


def _level_set_width(Vinv, L, axis):
    """Full width through the centre along `axis` of {L - x^T Vinv x / 2 >= 0},
    found by bisection on the density itself."""
    e = np.zeros(2)
    e[axis] = 1.0

    def f(r):
        d = r * e
        return L - 0.5 * d @ Vinv @ d

    lo, hi = 0.0, 1.0
    while f(hi) > 0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 2.0 * lo


def test_coverage_general_equals_bisected_level_set(orc):
    """Sec. 4.1 definition for rotated, anisotropic splats at any opacity:
    the smaller of the horizontal and vertical level-set widths, measured
    by bisection on the 2D density built from the oracle's 2D covariance."""
    cam = inputs.config1_camera()
    sc = inputs.single_level_scene(n=200, seed=3)
    cover, ux, uy, cov2d = orc.coverage64(sc, cam)
    for i in range(200):
        if cover[i] < 0:
            continue
        V = np.array([[cov2d[i, 0], cov2d[i, 1]], [cov2d[i, 1], cov2d[i, 2]]])
        L = math.log(255.0 * float(sc.opacity[i]))
        w = min(_level_set_width(np.linalg.inv(V), L, 0),
                _level_set_width(np.linalg.inv(V), L, 1))
        assert cover[i] == pytest.approx(w, rel=1e-9)


def test_projected_covariance_is_linearised_perspective(orc):
    """Sec. 3.1 (EWA splatting): V = J W Sigma W^T J^T with J the Jacobian
    of the pixel projection.  Pinned against a numerical Jacobian of
    (fx x/z + cx, fy y/z + cy) and scipy's quaternion -> matrix."""
    cams = inputs.orbit_cameras(3, seed=5, radius=4.0, width=320, height=240)
    sc = inputs.single_level_scene(n=300, seed=7)
    for cam in cams:
        cover, ux, uy, cov2d = orc.coverage64(sc, cam)
        R = cam.R.astype(np.float64)
        t = cam.t.astype(np.float64)
        for i in range(0, 300, 7):
            if cover[i] < 0:
                continue
            pc = R @ sc.mean[i].astype(np.float64) + t
            limx = 1.3 * 0.5 * cam.width / cam.fx
            limy = 1.3 * 0.5 * cam.height / cam.fy
            if abs(pc[0] / pc[2]) > limx or abs(pc[1] / pc[2]) > limy:
                continue

            def proj(p):
                return np.array([cam.fx * p[0] / p[2] + cam.cx,
                                 cam.fy * p[1] / p[2] + cam.cy])

            h = 1e-6
            J = np.stack([(proj(pc + h * e) - proj(pc - h * e)) / (2 * h)
                          for e in np.eye(3)], axis=1)
            w, x, y, z = sc.quat[i].astype(np.float64)
            Rq = Rotation.from_quat([x, y, z, w]).as_matrix()
            S = np.diag(np.exp(2.0 * sc.log_scale[i].astype(np.float64)))
            Sig = Rq @ S @ Rq.T
            V = J @ R @ Sig @ R.T @ J.T
            got = np.array([[cov2d[i, 0], cov2d[i, 1]], [cov2d[i, 1], cov2d[i, 2]]])
            np.testing.assert_allclose(got, V, rtol=1e-6, atol=1e-9 * np.abs(V).max())
            np.testing.assert_allclose([ux[i], uy[i]], proj(pc), rtol=1e-12)


def test_fp32_footprint_tracks_fp64(orc):
    """The fixed-order FP32 footprint stays within single-precision
    rounding of the FP64 definition (coverage, centre)."""
    cam = inputs.config2_camera()
    sc = inputs.multiscale_scene(n=20_000, seed=1)
    fp = orc.footprints(sc, cam, "all_levels")
    cover, ux, uy, _ = orc.coverage64(sc, cam)
    ok = (fp["valid"] == 1) & (cover > 0)
    assert ok.mean() > 0.99
    np.testing.assert_allclose(fp["cover"][ok], cover[ok], rtol=5e-5)
    np.testing.assert_allclose(fp["ux"][ok], ux[ok], rtol=0, atol=2e-4)
    np.testing.assert_allclose(fp["uy"][ok], uy[ok], rtol=0, atol=2e-4)


def test_enlargement_gives_coverage_ST_and_paper_bandwidth(orc):
    """Supplementary "Average Pooling and Enlargement" and Eq. 8: enlarging
    a Gaussian's scaling by S_T / S gives coverage S_T; for a unit-opacity
    Gaussian the enlarged 1-D Gaussian has 3 dB bandwidth 0.441 px^-1."""
    g = golden_constants()
    cam = inputs.config1_camera()
    sc = inputs.single_level_scene(n=500, seed=11)
    sc.opacity[:] = 1.0
    fp = orc.footprints(sc, cam, "all_levels")
    S = fp["cover"].astype(np.float64)
    ok = (fp["valid"] == 1) & (S > 0)
    big = sc.copy()
    big.log_scale += np.log(g["S_T"] / np.where(ok, S, 1.0))[:, None].astype(np.float32)
    fp2 = orc.footprints(big, cam, "all_levels")
    np.testing.assert_allclose(fp2["cover"][ok], g["S_T"], rtol=2e-5)
    # on-axis, axis-aligned: the narrow axis' pixel-space 1-D Gaussian
    one = one_gaussian([[0, 0, 0]], [-3.0, -2.0, -2.5], opacity=1.0)
    S1 = float(orc.coverage64(one, cam)[0][0])
    one.log_scale += np.float32(math.log(g["S_T"] / S1))
    s_px = cam.fx * math.exp(float(one.log_scale[0, 0])) / 3.0
    a = 1.0 / (2.0 * s_px ** 2)
    f3db = math.sqrt(a * math.log(math.sqrt(2.0))) / math.pi
    assert f3db == pytest.approx(g["f3dB_enlarged"], abs=5e-4)
    assert f3db < 0.5


# ------------------------------------------------------------------- blend

def test_single_isotropic_gaussian_closed_form(orc):
    """One isotropic Gaussian on the optical axis: its splat is isotropic
    with variance s_px^2 + 0.3, so pixel = rgb min(0.99, sigma
    exp(-r^2 / (2 (s_px^2 + 0.3)))) where that is >= 1/255, else bg."""
    cam = inputs.config1_camera(64, 64)
    for ls, op, rgb in [(-3.0, 0.8, (0.2, 0.5, 0.9)), (-4.5, 0.95, (1, 0, 0.5)),
                        (-2.0, 0.3, (0.7, 0.7, 0.1))]:
        sc = one_gaussian([[0, 0, 0]], [ls] * 3, opacity=op, rgb=rgb)
        r = orc.render(sc, cam, "all_levels")
        s_px = cam.fx * math.exp(ls) / 3.0
        var = s_px ** 2 + 0.3
        ys, xs = np.mgrid[0:64, 0:64] + 0.5
        r2 = (xs - 32.0) ** 2 + (ys - 32.0) ** 2
        g = op * np.exp(-r2 / (2 * var))
        alpha = np.minimum(0.99, g)
        alpha[g < 1 / 255] = 0.0
        want = alpha[None] * np.asarray(rgb, np.float64)[:, None, None]
        near = np.abs(g - 1 / 255) < 1e-5
        np.testing.assert_allclose(r["image"][:, ~near], want[:, ~near], atol=2e-6)
        np.testing.assert_allclose(r["final_t"][~near], 1 - alpha[~near], atol=2e-6)


def test_front_gaussian_wins(orc):
    """Front-to-back order by depth (Sec. 3.1): two nearly opaque Gaussians
    on the axis at z = 2 and z = 4; the nearer one's colour is blended
    first whatever the index order: red = a_f, green = (1 - a_f) a_b with
    each a = min(0.99, sigma exp(-r^2 / (2 (s_px^2 + 0.3))))."""
    cam = inputs.config1_camera(32, 32)
    for order in (0, 1):
        pos = [[0, 0, -1.0], [0, 0, 1.0]]
        rgb = np.array([[1, 0, 0], [0, 1, 0]], np.float32)
        if order:
            pos, rgb = pos[::-1], rgb[::-1].copy()
        sc = one_gaussian(pos, [-1.0] * 3, opacity=0.9999)
        sc.color = rgb
        r = orc.render(sc, cam, "all_levels")
        c = r["image"][:, 16, 16]
        r2 = 0.5                                   # pixel centre (16.5, 16.5)
        a = []
        for z in (2.0, 4.0):
            s_px = cam.fx * math.exp(float(sc.log_scale[0, 0])) / z
            a.append(min(0.99, 0.9999 * math.exp(-r2 / (2 * (s_px ** 2 + 0.3)))))
        assert c[0] == pytest.approx(a[0], rel=1e-6)
        assert c[1] == pytest.approx((1 - a[0]) * a[1], rel=1e-5)
        assert c[0] > 0.98 and c[1] < 0.02


def test_white_scene_telescopes(orc):
    """With every colour 1 and a black background, sum_k alpha_k T_k
    telescopes to 1 - T_final (Eq. 3 with incremental T)."""
    cam = inputs.config1_camera(128, 128)
    sc = inputs.single_level_scene(n=3000, seed=2)
    sc.color[:] = 1.0
    r = orc.render(sc, cam, "all_levels")
    np.testing.assert_allclose(r["image"][0], 1.0 - r["final_t"], atol=1e-12)
    assert np.all(r["final_t"] <= 1.0) and np.all(r["final_t"] >= 1e-4)
    # early termination happened somewhere, and T stops at >= 1e-4
    assert np.any(r["final_t"] < 1e-3)


def test_evaluation_counts(orc):
    """The per-pixel evaluation count (the work the raster roofline counts):
    every entry of the tile's list up to and including the one that ended
    the pixel, else the whole list.  The ending entry is a Gaussian with
    alpha >= 1/255 at the pixel that would bring the final T below 1e-4
    (Eq. 3, stop before it), it comes after the last blended entry, and the
    counts sum to the returned total."""
    cam = inputs.config1_camera(128, 96)
    sc = inputs.single_level_scene(n=12000, seed=5)
    r = orc.render(sc, cam, "all_levels")
    ne, nc, ft = r["n_eval"], r["n_contrib"].astype(np.int64), r["final_t"]
    off, idx, fp = r["offsets"], r["idx"], r["fp"]
    assert ne.sum() == r["evals"]
    lens = np.diff(off)
    ended = 0
    for y in range(cam.height):
        for x in range(cam.width):
            t = (y // 16) * cam.tiles_x + x // 16
            n = int(ne[y, x])
            assert nc[y, x] < n <= lens[t] or nc[y, x] == n == lens[t]
            if n == lens[t]:
                continue
            g = idx[off[t] + n - 1]
            dx, dy = x + 0.5 - float(fp["ux"][g]), y + 0.5 - float(fp["uy"][g])
            a, b, c = (float(v) for v in fp["conic"][g])
            power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
            alpha = min(0.99, float(sc.opacity[g]) * math.exp(power))
            assert power <= 0.0 and alpha >= 1.0 / 255.0
            assert ft[y, x] * (1.0 - alpha) < 1e-4
            ended += 1
    assert ended > 200


def test_brute_force_equals_tiled(orc):
    """Per-pixel blending of every selected Gaussian in one global depth
    order, with no tiles, equals the tiled render bit for bit wherever no
    Gaussian sits on the alpha threshold (the level-set box bounds every
    pixel a Gaussian can reach)."""
    for seed, deg, nl in [(0, -1, 1), (1, 3, 4), (2, 1, 2), (3, 0, 1)]:
        sc = inputs.tiny_scene(n=64, seed=seed, sh_degree=deg, n_levels=nl)
        cam = inputs.config1_camera(64, 64)
        cam.bg[:] = [0.1, 0.2, 0.3]
        for mode in ("all_levels", "selective"):
            if nl > 1:
                orc.calibrate(sc, inputs.orbit_cameras(4, seed=seed, radius=3.0,
                                                       width=64, height=64))
            t = orc.render(sc, cam, mode)
            b = orc.render_brute(sc, cam, mode)
            ok = (t["flags"] & 1) == 0
            ok &= (b["flags"] & 1) == 0
            assert ok.mean() > 0.97
            # the brute force path has no early stop flag; exclude T flips
            ok &= (t["flags"] & 2) == 0
            assert np.array_equal(t["image"][:, ok], b["image"][:, ok])
            assert np.array_equal(t["final_t"][ok], b["final_t"][ok])


def test_tile_lists_by_enumeration(orc):
    """Per-tile lists equal a direct enumeration: every selected Gaussian
    whose tile rectangle covers the tile, ordered by depth then index; and
    every pixel where a Gaussian reaches alpha >= 1/255 lies in its
    rectangle."""
    cam = inputs.config1_camera(80, 48)   # 5 x 3 tiles
    sc = inputs.tiny_scene(n=60, seed=4)
    sc.mean[::7, 2] = sc.mean[3, 2]       # equal depths -> index tie-break
    fp = orc.footprints(sc, cam, "all_levels")
    off, idx = orc.tile_lists(fp, cam)
    depth_f = fp["depth"].view(np.float32)
    for t in range(cam.tiles_x * cam.tiles_y):
        tx, ty = t % cam.tiles_x, t // cam.tiles_x
        members = [i for i in range(sc.n)
                   if fp["selected"][i] and fp["ntiles"][i] > 0
                   and fp["rect"][i][0] <= tx <= fp["rect"][i][2]
                   and fp["rect"][i][1] <= ty <= fp["rect"][i][3]]
        want = sorted(members, key=lambda i: (float(depth_f[i]), i))
        assert list(idx[off[t]:off[t + 1]]) == want
    ys, xs = np.mgrid[0:48, 0:80] + 0.5
    for i in range(sc.n):
        if not fp["valid"][i]:
            continue
        a, b, c = fp["conic"][i].astype(np.float64)
        dx, dy = xs - fp["ux"][i], ys - fp["uy"][i]
        g = sc.opacity[i] * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
        hit = g >= (1 / 255) * (1 + 1e-6)
        if not hit.any():
            continue
        x0, y0, x1, y1 = fp["rect"][i]
        tyx = np.stack([ys[hit] // 16, xs[hit] // 16])
        assert np.all((tyx[1] >= x0) & (tyx[1] <= x1) & (tyx[0] >= y0) & (tyx[0] <= y1))


def test_single_level_selective_reduces_to_all_levels(orc):
    """Sec. 4.1 exemptions: with one level the finest level is also the
    coarsest, so selective rendering keeps every valid Gaussian and the
    image equals the single-scale render."""
    cam = inputs.config1_camera()
    sc = inputs.single_level_scene(n=10_000, seed=0)
    rng = np.random.default_rng(9)
    sc.s_max[:] = rng.uniform(0.0, 5.0, sc.n)
    sc.s_min[:] = rng.uniform(5.0, 50.0, sc.n)
    a = orc.render(sc, cam, "all_levels")
    s = orc.render(sc, cam, "selective")
    assert np.array_equal(a["fp"]["selected"], s["fp"]["selected"])
    assert np.array_equal(a["idx"], s["idx"])
    assert np.array_equal(a["image"], s["image"])


def test_update_range_eq5(orc):
    """Eq. 5 with the paper's decays: first update from (0, inf) gives S;
    later updates decay the stored bounds by 0.95 / 1.05 before comparing.
    Only the level being rendered at its creation scale is updated."""
    cam = inputs.config1_camera()
    sc = one_gaussian([[0, 0, 0], [0.1, 0, 0]], [-3.0, -3.0, -3.0],
                      level=[2, 1], n_levels=2)
    orc.update_range(sc, cam, 2)
    S = float(orc.footprints(sc, cam, "all_levels")["cover"][0])
    assert sc.s_max[0] == np.float32(S) and sc.s_min[0] == np.float32(S)
    assert sc.s_max[1] == 0.0 and np.isinf(sc.s_min[1])
    sc.s_max[0], sc.s_min[0] = 2 * S, 0.5 * S
    orc.update_range(sc, cam, 2)
    assert sc.s_max[0] == np.float32(0.95) * np.float32(2 * S)
    assert sc.s_min[0] == np.float32(1.05) * np.float32(0.5 * S)
    sc.s_max[0], sc.s_min[0] = S / 2, S * 2
    orc.update_range(sc, cam, 2)
    assert sc.s_max[0] == np.float32(S) and sc.s_min[0] == np.float32(S)


# --------------------------------------------------------------------- SH

def test_sh_basis_matches_scipy_and_is_orthonormal(orc):
    """Real SH built from scipy.special.sph_harm_y (complex, Condon-Shortley
    phase) agree with the oracle's recurrence; Gauss-Legendre x uniform
    quadrature shows orthonormality to degree 3."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(0)
    for _ in range(20):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        theta = math.acos(d[2])
        phi = math.atan2(d[1], d[0])
        got = orc.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                Y = sph_harm_y(l, abs(m), theta, phi)
                if m == 0:
                    want = Y.real
                elif m > 0:
                    want = math.sqrt(2) * (-1) ** m * Y.real
                else:
                    want = math.sqrt(2) * (-1) ** m * Y.imag
                assert got[l * l + l + m] == pytest.approx(want, abs=1e-12)
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for z, wz in zip(xg, wg):
        for k in range(nphi):
            p = 2 * math.pi * k / nphi
            s = math.sqrt(1 - z * z)
            Y = orc.sh_basis(3, [s * math.cos(p), s * math.sin(p), z])
            G += np.outer(Y, Y) * wz * (2 * math.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_colour_is_view_dependent_and_dc_offset(orc):
    """DC-only coefficients give a view-independent colour Y_00 f + 0.5."""
    sc = inputs.tiny_scene(n=10, seed=1, sh_degree=3)
    sc.color[:, 1:, :] = 0.0
    cam = inputs.config1_camera(64, 64)
    rgb = orc.colors(sc, cam)
    want = np.maximum(0.0, 0.5 / math.sqrt(math.pi) * sc.color[:, 0, :].astype(np.float64) + 0.5)
    np.testing.assert_allclose(rgb, want, rtol=1e-12)


def _cartesian_sh(k, d):
    """Textbook real spherical harmonics in Cartesian form (unit vector d =
    (x, y, z), no Condon-Shortley phase, k = l^2 + l + m) for the
    coefficients the colour pins use."""
    x, y, z = d
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    c33 = 0.25 * math.sqrt(35.0 / (2.0 * math.pi))
    c30 = 0.25 * math.sqrt(7.0 / math.pi)
    c31 = 0.25 * math.sqrt(21.0 / (2.0 * math.pi))
    table = {
        1: c1 * y,                                   # l = 1, m = -1
        2: c1 * z,                                   # l = 1, m = 0
        3: c1 * x,                                   # l = 1, m = 1
        9: c33 * y * (3 * x * x - y * y),            # l = 3, m = -3
        12: c30 * z * (5 * z * z - 3),               # l = 3, m = 0
        13: c31 * x * (5 * z * z - 1),               # l = 3, m = 1
        15: c33 * x * (x * x - 3 * y * y),           # l = 3, m = 3
    }
    return table[k]


@pytest.mark.parametrize("k", [1, 2, 3, 9, 12, 13, 15])
def test_sh_colour_single_coefficient_direction_and_layout(orc, k):
    """A lone SH coefficient f at index k of channel c gives colour
    max(0, 0.5 + f Y_k(d)) in channel c and 0.5 in the others, with d the
    unit direction from the camera centre to the mean.  Placing the mean on
    the other side of the camera flips d and so the sign of Y_k for the odd
    degrees 1 and 3: a colour taken along campos - mean, or a coefficient
    read as [k][i][c] or [i][c][k], fails."""
    cam = inputs.config1_camera(64, 64)
    campos = np.asarray(cam.campos, np.float64)
    for deg in (1, 3):
        if k >= (deg + 1) ** 2:
            continue
        K = (deg + 1) ** 2
        for ch in range(3):
            for sign in (1.0, -1.0):
                off = sign * np.array([0.9, -0.4, 0.6])
                pos = (campos + off).astype(np.float32)[None]
                sc = one_gaussian(pos, [-3.0] * 3)
                sc.sh_degree = deg
                sc.color = np.zeros((1, K, 3), np.float32)
                f = np.float32(0.37)
                sc.color[0, k, ch] = f
                rgb = orc.colors(sc, cam)[0]
                d = pos[0].astype(np.float64) - campos
                d /= np.linalg.norm(d)
                want = np.full(3, 0.5)
                want[ch] = max(0.0, 0.5 + float(f) * _cartesian_sh(k, d))
                np.testing.assert_allclose(rgb, want, rtol=0, atol=1e-7)
                # the odd degrees change sign with the direction
                assert abs(_cartesian_sh(k, d)) > 0.01


def test_forward64_full_isotropic_closed_form(orc):
    """The FP64 forward that the gradient differentiates (FP64 projection,
    fixed tile lists): one isotropic Gaussian on the optical axis at depth
    3 renders rgb min(0.99, sigma exp(-r^2 / (2 (s_px^2 + 0.3)))) where that
    is >= 1/255, with s_px = f e^s / 3 and r the distance to the image
    centre; with SH degree 0 the colour is 0.5 + f_0 / (2 sqrt(pi))."""
    cam = inputs.config1_camera(64, 64)
    for ls, op, dc in [(-3.0, 0.8, (0.2, -0.5, 0.9)), (-4.5, 0.95, (1.0, 0.0, 0.5)),
                       (-2.0, 0.3, (0.7, 0.7, -1.5))]:
        sc = one_gaussian([[0, 0, 0]], [ls] * 3, opacity=op)
        sc.sh_degree = 0
        sc.color = np.asarray(dc, np.float32).reshape(1, 1, 3)
        fp = orc.footprints(sc, cam, "all_levels")
        off, idx = orc.tile_lists(fp, cam)
        r = orc.forward64(sc, cam, off, idx)
        s_px = cam.fx * math.exp(ls) / 3.0
        ys, xs = np.mgrid[0:64, 0:64] + 0.5
        r2 = (xs - 32.0) ** 2 + (ys - 32.0) ** 2
        g = op * np.exp(-r2 / (2 * (s_px ** 2 + 0.3)))
        alpha = np.where(g >= 1 / 255, np.minimum(0.99, g), 0.0)
        rgb = np.maximum(0.0, 0.5 + np.asarray(dc, np.float64) / (2 * math.sqrt(math.pi)))
        want = alpha[None] * rgb[:, None, None]
        near = np.abs(g - 1 / 255) < 1e-6
        # the camera pose and the inputs are FP32 values: about 1e-8 relative
        np.testing.assert_allclose(r["image"][:, ~near], want[:, ~near], rtol=0, atol=1e-7)
        np.testing.assert_allclose(r["final_t"][~near], 1 - alpha[~near], rtol=0, atol=1e-7)
        assert (alpha > 0).sum() >= 12


@pytest.mark.parametrize("seed,deg,nl,mode", [(0, -1, 1, "all_levels"), (1, 3, 4, "selective"),
                                              (2, 1, 2, "all_levels"), (5, 3, 1, "all_levels")])
def test_forward64_full_matches_footprint_render(orc, seed, deg, nl, mode):
    """The FP64 forward (FP64 projection of every splat) and the renderer
    whose splats come from the FP32 footprint produce the same image: they
    differ only by the rounding of the splat parameters to FP32, far below
    the 2e-4 tolerance, and on pixels whose decisions sit away from the
    thresholds they take the same contributors.  A Jacobian or colour slip
    in the FP64 projection that its own finite differences cannot see (it
    is shared by the forward and the gradient) fails here."""
    sc = inputs.tiny_scene(n=64, seed=seed, sh_degree=deg, n_levels=nl)
    cam = inputs.config1_camera(64, 64)
    cam.bg[:] = [0.1, 0.2, 0.3]
    if nl > 1:
        orc.calibrate(sc, inputs.orbit_cameras(4, seed=seed, radius=3.0, width=64, height=64))
    t = orc.render(sc, cam, mode)
    f = orc.forward64(sc, cam, t["offsets"], t["idx"])
    ok = t["flags"] == 0
    assert ok.mean() > 0.97
    # both images include the background T bg
    np.testing.assert_allclose(f["image"][:, ok], t["image"][:, ok], rtol=0, atol=1e-5)
    np.testing.assert_allclose(f["final_t"][ok], t["final_t"][ok], rtol=0, atol=1e-5)
    np.testing.assert_array_equal(f["n_contrib"][ok], t["n_contrib"][ok])
    assert np.abs(t["image"] - t["final_t"][None] * 0.2).max() > 0.05   # something is drawn
