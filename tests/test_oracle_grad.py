"""Pins of the oracle's analytic FP64 gradient (or_grad64) against central
finite differences of its FP64 forward (or_forward64_full) on tiny scenes.

The loss is L = sum(w * image) for a seeded random weight image w, so
dL/dimage = w.  Tile lists are held fixed (as in a training step).  A
parameter whose +-h perturbation changes any pixel's contributor signature
(a threshold decision flips inside the step) is excluded and counted.
"""
import numpy as np
import pytest

from paper_2311_17089_gb300 import inputs

# (step, relative): relative steps scale with max(1, |theta|); log-scales
# take an absolute step (it is already a relative change of the scale)
STEPS = {"mean": (1e-4, True), "log_scale": (1e-4, False), "quat": (1e-4, True),
         "opacity": (1e-4, True), "color": (1e-3, True)}


def _loss_and_sig(orc, sc, cam, off, idx, w):
    r = orc.forward64(sc, cam, off, idx)
    return float(np.sum(w * r["image"])), (r["n_contrib"].copy(), r["n_blend"].copy())


def _fd_check(orc, sc, cam, mode, rng, per_array=12):
    fp = orc.footprints(sc, cam, mode)
    off, idx = orc.tile_lists(fp, cam)
    w = rng.standard_normal((3, cam.height, cam.width))
    g = orc.grad64(sc, cam, off, idx, w)
    _, sig0 = _loss_and_sig(orc, sc, cam, off, idx, w)
    checked = excluded = 0
    worst = 0.0
    for name, (h, relative) in STEPS.items():
        arr = getattr(sc, name)
        grad = g[name].reshape(arr.shape)
        flat_g = grad.reshape(-1)
        cand = np.nonzero(np.abs(flat_g) > 1e-9 * (np.abs(flat_g).max() + 1e-30))[0]
        if len(cand) == 0:
            continue
        pick = rng.choice(cand, min(per_array, len(cand)), replace=False)
        scale = np.abs(flat_g).max()
        for j in pick:
            flat = arr.reshape(-1)
            th = flat[j]
            step = h * max(1.0, abs(float(th))) if relative else h
            tp = np.float32(th + step)
            tm = np.float32(th - step)
            flat[j] = tp
            lp, sp = _loss_and_sig(orc, sc, cam, off, idx, w)
            flat[j] = tm
            lm, sm = _loss_and_sig(orc, sc, cam, off, idx, w)
            flat[j] = th
            if not all(np.array_equal(a, b) for a, b in zip(sp + sm, sig0 + sig0)):
                excluded += 1
                continue
            fd = (lp - lm) / (float(tp) - float(tm))
            err = abs(fd - flat_g[j])
            tol = 1e-3 * max(abs(fd), abs(flat_g[j])) + 1e-6 * scale
            worst = max(worst, err / (tol + 1e-300))
            assert err <= tol, (name, j, fd, flat_g[j])
            checked += 1
    return checked, excluded, worst


@pytest.mark.parametrize("seed,deg,nl,mode", [(0, -1, 1, "all_levels"), (1, 3, 4, "selective"),
                                               (2, 1, 2, "all_levels"), (3, 2, 1, "all_levels")])
def test_oracle_gradient_matches_finite_differences(orc, seed, deg, nl, mode):
    sc = inputs.tiny_scene(n=64, seed=seed, sh_degree=deg, n_levels=nl)
    cam = inputs.config1_camera(64, 64)
    cam.bg[:] = [0.3, 0.1, 0.2]
    if nl > 1:
        orc.calibrate(sc, inputs.orbit_cameras(4, seed=seed, radius=3.0, width=64, height=64))
    checked, excluded, worst = _fd_check(orc, sc, cam, mode, np.random.default_rng(seed))
    assert checked >= 40 and excluded <= checked // 4, (checked, excluded)


def test_oracle_gradient_of_single_gaussian_closed_form(orc):
    """One isotropic Gaussian on the axis, weight 1 on the red channel:
    L = sum_p min(0.99, sigma e^power) r, so dL/dr = sum_p alpha_p and
    dL/dsigma = sum_p e^power_p r over unclamped pixels."""
    sc = inputs.Scene(np.zeros((1, 3), np.float32), np.full((1, 3), -2.0, np.float32),
                      np.array([[1, 0, 0, 0]], np.float32), np.array([0.6], np.float32),
                      np.array([[0.7, 0.2, 0.1]], np.float32), np.ones(1, np.uint8), 1, -1,
                      np.zeros(1, np.float32), np.full(1, np.inf, np.float32))
    cam = inputs.config1_camera(48, 48)
    fp = orc.footprints(sc, cam, "all_levels")
    off, idx = orc.tile_lists(fp, cam)
    w = np.zeros((3, 48, 48))
    w[0] = 1.0
    g = orc.grad64(sc, cam, off, idx, w)
    s_px = cam.fx * np.exp(-2.0) / 3.0
    var = s_px ** 2 + 0.3
    ys, xs = np.mgrid[0:48, 0:48] + 0.5
    e = np.exp(-((xs - 24) ** 2 + (ys - 24) ** 2) / (2 * var))
    a = 0.6 * e
    keep = a >= 1 / 255
    assert g["color"][0, 0] == pytest.approx(float(a[keep].sum()), rel=1e-5)
    assert g["opacity"][0] == pytest.approx(float((e * 0.7)[keep].sum()), rel=1e-5)
    # symmetric splat on the optical axis: no pull sideways
    assert abs(g["mean"][0, 0]) < 1e-6 * abs(g["opacity"][0]) + 1e-9
