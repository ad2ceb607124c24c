"""Pins of the oracle's visibility filter V (Eq. meth::sparse_beta: 1 for a
primitive seen from the current viewpoint), read as the frustum test of the
primitive's mean.  The FP32 decision is checked against an independent
angular formulation in FP64 away from the planes, and against hand-placed
points (on the axis, behind the camera, exactly on a side plane)."""
import math

import numpy as np
import pytest

from paper_2601_16736_gb300 import synth


def _ident_cam(tanx=0.5, tany=0.25, zn=0.5, zf=50.0):
    return np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, tanx, tany, zn, zf], np.float32)


def test_hand_placed_points(orc):
    cam = _ident_cam()
    pts = np.array([
        [0.0, 0.0, 10.0],      # on the optical axis -> visible
        [0.0, 0.0, -10.0],     # behind the camera -> not
        [4.0, 0.0, 10.0],      # x / z = 0.4 < 0.5 -> visible
        [6.0, 0.0, 10.0],      # x / z = 0.6 > 0.5 -> not
        [0.0, -2.0, 10.0],     # |y| / z = 0.2 < 0.25 -> visible
        [0.0, 3.0, 10.0],      # 0.3 > 0.25 -> not
        [0.0, 0.0, 0.25],      # nearer than z_near -> not
        [0.0, 0.0, 60.0],      # beyond z_far -> not
        [5.0, 0.0, 10.0],      # exactly on the right plane (exact in FP32) -> visible, margin 0
        [0.0, 0.0, 0.5],       # exactly on the near plane -> visible
    ], np.float32)
    mask = orc.visibility_f32(pts, cam)
    assert mask.tolist() == [1, 0, 1, 0, 1, 0, 0, 0, 1, 1]
    margin, mask64 = orc.frustum_margin_f64(pts, cam)
    assert margin[8] == 0.0 and margin[9] == 0.0
    assert mask64.tolist() == mask.tolist()


def test_look_at_camera_centres_target(orc):
    cam = synth.look_at_camera((10.0, 0.0, 0.0))
    R = cam[:9].reshape(3, 3).astype(np.float64)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
    p = R @ np.zeros(3) + cam[9:12]
    np.testing.assert_allclose(p, [0, 0, 10], atol=1e-5)
    # world up (+z) maps to image up (-y in OpenCV axes)
    assert (R @ np.array([0, 0, 1.0]))[1] < -0.99


def test_against_angular_formulation(orc):
    """Independent FP64 formulation: visible iff z in [near, far] and the
    horizontal / vertical view angles atan2(x, z), atan2(y, z) are within the
    half field of view.  Rows farther than 1e-4 from every plane must agree
    with the FP32 decision; nearer ones are the only ones allowed to differ."""
    g = synth.scene_blobs(200_000, 81, extent=12.5)
    cams = synth.ring_cameras(8, (-30.0, 0.0, 30.0))
    for cam in cams:
        xyz = g["xyz"]
        mask = orc.visibility_f32(xyz, cam)
        margin, mask64 = orc.frustum_margin_f64(xyz, cam)
        R = cam[:9].reshape(3, 3).astype(np.float64)
        p = xyz.astype(np.float64) @ R.T + cam[9:12].astype(np.float64)
        hx = math.atan(float(cam[12]))
        hy = math.atan(float(cam[13]))
        ang = ((p[:, 2] >= cam[14]) & (p[:, 2] <= cam[15]) &
               (np.abs(np.arctan2(p[:, 0], p[:, 2])) <= hx) & (np.abs(np.arctan2(p[:, 1], p[:, 2])) <= hy))
        far = np.abs(margin) > 1e-4
        assert np.array_equal(ang[far], mask[far].astype(bool))
        assert np.array_equal(mask64[far], mask[far])
        # the FP64 sign convention matches the angular test everywhere off the planes
        assert np.array_equal(mask64[np.abs(margin) > 1e-9].astype(bool), ang[np.abs(margin) > 1e-9])


def test_nan_mean_is_invisible(orc):
    cam = _ident_cam()
    pts = np.array([[np.nan, 0, 10], [0, np.nan, 10], [0, 0, np.nan]], np.float32)
    assert orc.visibility_f32(pts, cam).tolist() == [0, 0, 0]


def _near_plane_means(cam, n, rng):
    """Means at relative distances 1e-8 .. 1e-4 from the side planes of `cam`."""
    R = cam[:9].reshape(3, 3).astype(np.float64)
    t = cam[9:12].astype(np.float64)
    tx, ty = float(cam[12]), float(cam[13])
    pz = rng.uniform(0.5, 40.0, n)
    side = rng.integers(0, 4, n)
    d = rng.normal(0, 1, n) * 10.0 ** rng.uniform(-8, -4, n)
    sgn = np.where(side % 2 == 0, 1.0, -1.0)
    px = np.where(side < 2, sgn * pz * tx * (1 + d), rng.uniform(-1, 1, n) * pz * tx)
    py = np.where(side >= 2, sgn * pz * ty * (1 + d), rng.uniform(-1, 1, n) * pz * ty)
    return ((np.stack([px, py, pz], 1) - t) @ R).astype(np.float32)


def test_fp32_band_bounds_every_fp32_disagreement(orc):
    """The FP32 evaluation of the frustum test differs from the FP64
    decision only within the band derived from the inner-product rounding
    bound, and the band is tight to within a small factor (the worst
    disagreement reaches a sizeable fraction of it).  Many disagreements lie
    beyond 1e-6 of a plane, so an FP32 decision alone cannot meet a 1e-6
    tolerance: the kernels re-decide inside the band in FP64."""
    rng = np.random.default_rng(1300)
    worst, beyond = 0.0, 0
    for cam in synth.ring_cameras(4, (-30.0, 0.0, 30.0)) + [_ident_cam(0.7, 0.3, 0.5, 60.0)]:
        xyz = _near_plane_means(cam, 100_000, rng)
        f32 = orc.visibility_f32(xyz, cam)
        margin, f64 = orc.frustum_margin_f64(xyz, cam)
        band = orc.frustum_fp32_band(xyz, cam)
        differ = f32 != f64
        assert differ.sum() > 100
        assert np.all(np.abs(margin[differ]) <= band[differ])
        worst = max(worst, float((np.abs(margin[differ]) / band[differ]).max()))
        beyond += int((np.abs(margin[differ]) > 1e-6).sum())
        # away from the band both evaluations agree
        assert np.array_equal(f32[np.abs(margin) > band], f64[np.abs(margin) > band])
    assert worst > 0.1, f"band far looser than the observed error ({worst:.3f})"
    assert beyond > 0


def test_fp32_band_closed_form(orc):
    """The band of one mean, by hand: identity rotation, t = 0, mu = (1, 2, 10),
    tan = (0.5, 0.25): S = (1, 2, 10), e = gamma_4 S; side x gives
    (1 + 0.5 * 10) gamma_4 + u * 0.5 * (10 + 10 gamma_4), over sqrt(1.25)."""
    cam = _ident_cam(0.5, 0.25, 0.5, 50.0)
    u = 2.0 ** -24
    g4 = 4 * u / (1 - 4 * u)
    bx = (g4 * 1 + 0.5 * g4 * 10 + u * 0.5 * (10 + g4 * 10)) / math.sqrt(1.25)
    by = (g4 * 2 + 0.25 * g4 * 10 + u * 0.25 * (10 + g4 * 10)) / math.sqrt(1.0625)
    want = max(bx, by, g4 * 10) + 1e-12 * 11
    got = orc.frustum_fp32_band(np.array([[1.0, 2.0, 10.0]], np.float32), cam)[0]
    assert got == pytest.approx(want, rel=1e-12)
