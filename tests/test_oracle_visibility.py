"""Pins of the oracle's visibility filter V (Eq. meth::sparse_beta: 1 for a
primitive seen from the current viewpoint), read as the frustum test of the
primitive's mean.  The FP32 decision is checked against an independent
angular formulation in FP64 away from the planes, and against hand-placed
points (on the axis, behind the camera, exactly on a side plane)."""
import math

import numpy as np

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
