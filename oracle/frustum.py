"""FP64 CPU oracle for the visibility mask of the scene-scale training step.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the benchmark).

The paper renders with a pinhole camera and evaluates the appearance model for
the primitives a frame sees (Sec. 5.2: one evaluation per primitive per frame).
A primitive is visible when its centre lies in the symmetric frustum of the
camera: with p = R (mu - c) in camera coordinates (rows of R: right, up,
forward), p_z > near and |p_x| <= t p_z and |p_y| <= t p_z, t = tan(fov/2).
"""
import numpy as np


def camera_coords(means, rot, center):
    return (np.asarray(means, dtype=np.float64) - np.asarray(center, dtype=np.float64)) @ \
        np.asarray(rot, dtype=np.float64).T


def visible(means, rot, center, tan_half_fov, near=0.0):
    """Boolean mask of primitives inside the frustum."""
    p = camera_coords(means, rot, center)
    z = p[:, 2]
    t = float(tan_half_fov)
    return (z > near) & (np.abs(p[:, 0]) <= t * z) & (np.abs(p[:, 1]) <= t * z)


def boundary_margin(means, rot, center, tan_half_fov, near=0.0):
    """Distance (in camera-space units) of each centre to the nearest frustum face test;
    decisions within a few float32 ulps of 0 may legitimately differ between precisions."""
    p = camera_coords(means, rot, center)
    z = p[:, 2]
    t = float(tan_half_fov)
    return np.minimum.reduce([np.abs(z - near), np.abs(t * z - np.abs(p[:, 0])), np.abs(t * z - np.abs(p[:, 1]))])
