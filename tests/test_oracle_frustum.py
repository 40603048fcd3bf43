"""Pins of the visibility oracle (oracle/frustum.py) against cases the pinhole
geometry fixes by hand.

A centre mu is visible iff, with p = R (mu - c) (rows of R: right, up, forward),
p_z > near and |p_x| <= t p_z and |p_y| <= t p_z, t = tan(fov/2): faces are
inclusive, the near plane exclusive. The cases below would fail for R applied
transposed, for a strict inequality on a face, for an inclusive near plane, for a
dropped near test, and for a camera centre that is not subtracted.
"""
import math

import numpy as np
import pytest

from oracle import frustum as ofr
from paper_2606_09794_gb300 import inputs

EYE = np.eye(3)


def test_points_on_each_face_are_inside():
    # camera at the origin looking along +z, 90 degree field of view (t = 1)
    pts = np.array([[1.0, 0.0, 1.0], [-1.0, 0.0, 1.0], [0.0, 1.0, 1.0], [0.0, -1.0, 1.0],
                    [2.0, 2.0, 2.0], [-3.0, 3.0, 3.0]])
    assert ofr.visible(pts, EYE, np.zeros(3), 1.0).all()
    np.testing.assert_array_equal(ofr.boundary_margin(pts, EYE, np.zeros(3), 1.0), np.zeros(len(pts)))


def test_points_just_outside_a_face_are_outside():
    eps = 1e-12
    pts = np.array([[1.0 + eps, 0.0, 1.0], [0.0, -(1.0 + eps), 1.0], [2.0, 2.0 + 2 * eps, 2.0]])
    assert not ofr.visible(pts, EYE, np.zeros(3), 1.0).any()


def test_near_plane_and_behind():
    c = np.zeros(3)
    pts = np.array([[0.0, 0.0, -1.0],    # behind the camera
                    [0.0, 0.0, 0.0],     # at the centre (p_z = 0 = near)
                    [0.0, 0.0, 0.5],     # exactly at near = 0.5: not drawn
                    [0.0, 0.0, 0.5 + 1e-12],
                    [0.1, 0.1, 0.75]])
    np.testing.assert_array_equal(ofr.visible(pts, EYE, c, 1.0, near=0.5), [False, False, False, True, True])
    # without a near plane the centre itself is still not visible (p_z > 0 is strict)
    np.testing.assert_array_equal(ofr.visible(pts, EYE, c, 1.0), [False, False, True, True, True])
    # the margin of a centre on the axis is its distance to the near plane
    np.testing.assert_allclose(ofr.boundary_margin(pts[3:4] + [0, 0, 1.5], EYE, c, 1.0, near=0.5), [1.5 + 1e-12])


def test_camera_centre_is_subtracted():
    c = np.array([1.0, 2.0, 3.0])
    pts = np.array([[1.0, 2.0, 4.0],      # one unit in front of the camera
                    [0.0, 0.0, 1.0],      # in front of the origin, behind this camera
                    [1.9, 2.0, 4.0]])     # |p_x| = 0.9 <= 0.5 * 1? no: t = 0.5 -> limit 0.5
    np.testing.assert_array_equal(ofr.visible(pts, EYE, c, 0.5), [True, False, False])


def test_rotated_camera_by_hand():
    # camera looking along +x with up = +z: rows (right, up, forward) of R
    right, up, fwd = np.array([0.0, -1.0, 0.0]), np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    R = np.stack([right, up, fwd])
    c = np.zeros(3)
    t = math.tan(math.radians(30.0))
    pts = np.array([[5.0, 0.0, 0.0],       # on the forward axis: visible
                    [-5.0, 0.0, 0.0],      # behind
                    [5.0, 5 * t, 0.0],     # on the left face (p_x = -5 t): visible
                    [5.0, 0.0, -5 * t],    # on the bottom face (p_y = -5 t): visible
                    [0.0, 0.0, 5.0],       # straight up (p_z = 0): not visible
                    [5.0, 0.0, 3.0]])      # above the top face
    np.testing.assert_array_equal(ofr.visible(pts, R, c, t), [True, False, True, True, False, False])
    p = ofr.camera_coords(pts, R, c)
    np.testing.assert_allclose(p[0], [0.0, 0.0, 5.0])
    np.testing.assert_allclose(p[2], [-5 * t, 0.0, 5.0], atol=1e-15)
    np.testing.assert_allclose(p[3], [0.0, -5 * t, 5.0], atol=1e-15)


def test_rotation_is_not_applied_transposed():
    # a rotation that is not symmetric: 60 degrees about z, then the camera looks along
    # its third row. A point on the forward axis is visible; under R^T it would not be.
    a = math.radians(60.0)
    Rz = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])   # forward row = +y rotated
    R = Rx @ Rz
    assert not np.allclose(R, R.T)
    fwd = R[2]
    mu = 4.0 * fwd + 0.1 * R[0]       # slightly right of the axis
    assert ofr.visible(mu[None], R, np.zeros(3), 0.2)[0]
    assert not ofr.visible(mu[None], R.T, np.zeros(3), 0.2)[0]
    np.testing.assert_allclose(ofr.camera_coords(mu[None], R, np.zeros(3))[0], [0.1, 0.0, 4.0], atol=1e-14)


def test_boundary_margin_is_the_distance_to_the_nearest_test():
    pts = np.array([[0.5, 0.2, 2.0], [-0.5, 1.9, 2.0], [0.0, 0.0, 0.3]])
    # |z - near|, |t z - |p_x||, |t z - |p_y||  with t = 1, near = 0.1
    expect = [min(1.9, 1.5, 1.8), min(1.9, 1.5, 0.1), min(0.2, 0.3, 0.3)]
    np.testing.assert_allclose(ofr.boundary_margin(pts, EYE, np.zeros(3), 1.0, near=0.1), expect, rtol=1e-14)


@pytest.mark.parametrize("j", range(8))
def test_ring_cameras_see_the_origin_and_not_behind(j):
    """The workload's ring cameras (orthonormal rows, looking at the origin): the origin
    is on the forward axis, a point twice as far behind the camera is not visible."""
    sc = inputs.shell_scene(2000, 1, 5, fov_sample=2000)
    cam = sc.cameras[j]
    R = np.asarray(cam.rot, dtype=np.float64)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
    c = np.asarray(cam.center, dtype=np.float64)
    behind = c + (c - 0.0)
    v = ofr.visible(np.stack([np.zeros(3), behind]), R, c, cam.tan_half_fov)
    np.testing.assert_array_equal(v, [True, False])
    p = ofr.camera_coords(np.zeros((1, 3)), R, c)[0]
    np.testing.assert_allclose(p[:2], [0.0, 0.0], atol=1e-6)
    np.testing.assert_allclose(p[2], np.linalg.norm(c), rtol=1e-6)
