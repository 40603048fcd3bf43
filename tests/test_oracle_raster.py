"""Pins of the FP64 compositing oracle (oracle/raster.py): closed forms for one
primitive and for opaque stacks, depth order, the pinhole projection against a
camera matrix, the EWA covariance against a numerical Jacobian, the footprint
bound, and the backward against finite differences."""
import math

import numpy as np
import pytest

from oracle import raster as orr

W, H = 40, 30


def _cam(centre=(0.0, 0.0, -4.0), tan=0.4):
    return orr.camera(np.eye(3), centre, W, H, tan)


def _scene(n, seed, spread=1.0, big=False):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-spread, spread, (n, 3))
    scales = np.exp(rng.uniform(-2.5, -1.2 if big else -1.8, (n, 3)))
    quats = rng.normal(size=(n, 4))
    opacity = rng.uniform(0.05, 0.98, n)
    colours = rng.uniform(0, 1, (n, 3))
    return means, scales, quats, opacity, colours


def test_single_isotropic_primitive_closed_form():
    """One isotropic primitive on the optical axis at distance d: Sigma' = ((fx s / d)^2 + 0.3) I,
    so every pixel is c sigma exp(-|delta|^2 / (2 v)) where that is >= 1/255, else 0."""
    cam = _cam()
    s, d, sig, c = 0.15, 4.0, 0.8, np.array([0.2, 0.5, 0.9])
    img, T = orr.render(np.zeros((1, 3)), np.full((1, 3), s), [[1, 0, 0, 0]], [sig], c[None], cam, W, H)
    v = (cam["fx"] * s / d) ** 2 + orr.LOWPASS
    jj, ii = np.mgrid[0:H, 0:W]
    r2 = (ii + 0.5 - cam["cx"]) ** 2 + (jj + 0.5 - cam["cy"]) ** 2
    a = sig * np.exp(-r2 / (2 * v))
    a = np.where(a >= orr.ALPHA_MIN, a, 0.0)
    np.testing.assert_allclose(img, a[..., None] * c, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(T, 1.0 - a, rtol=1e-12)


def test_depth_order_not_index_order():
    """Two primitives on the axis: the nearer one is composited first whatever its index."""
    cam = _cam()
    means = np.array([[0.0, 0, 1.0], [0.0, 0, -1.0]])       # index 1 is nearer to the camera
    sc = np.full((2, 3), 0.3)
    q = [[1, 0, 0, 0]] * 2
    op = [0.6, 0.7]
    col = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    img, _ = orr.render(means, sc, q, op, col, cam, W, H, pixels=np.array([[W // 2, H // 2]]))
    _, m2, s2, _ = orr.project(means, sc, q, cam)
    a = [min(0.99, op[k] * math.exp(-0.5 * (np.array([W // 2 + 0.5, H // 2 + 0.5]) - m2[k])
                                     @ np.linalg.solve(s2[k], np.array([W // 2 + 0.5, H // 2 + 0.5]) - m2[k])))
         for k in range(2)]
    want = col[1] * a[1] + col[0] * a[0] * (1 - a[1])
    np.testing.assert_allclose(img[0], want, rtol=1e-12)
    img2, _ = orr.render(means[::-1], sc, q, op[::-1], col[::-1], cam, W, H, pixels=np.array([[W // 2, H // 2]]))
    np.testing.assert_allclose(img2, img, rtol=1e-14)


def test_opaque_stack_stops_early():
    """Five coincident-footprint layers with alpha = 0.95 at the centre pixel: T goes
    1, 0.05, 0.0025, 1.25e-4; the fourth layer would take T below 1e-4, so exactly three count."""
    cam = _cam()
    n = 5
    means = np.stack([np.zeros(n), np.zeros(n), np.linspace(-1, 1, n)], axis=1)
    big = np.full((n, 3), 2.0)                       # nearly flat kernel at the centre pixel
    cx = np.array([[W // 2, H // 2]])
    _, m2, s2, _ = orr.project(means, big, [[1, 0, 0, 0]] * n, cam)
    delta = np.array([W // 2 + 0.5, H // 2 + 0.5]) - m2
    rho = np.exp(-0.5 * np.einsum("ni,nij,nj->n", delta, np.linalg.inv(s2), delta))
    op = 0.95 / rho
    col = np.eye(3)[np.arange(n) % 3]
    img, T = orr.render(means, big, [[1, 0, 0, 0]] * n, op, col, cam, W, H, pixels=cx)
    want = col[0] * 0.95 + col[1] * 0.95 * 0.05 + col[2] * 0.95 * 0.0025
    np.testing.assert_allclose(img[0], want, rtol=1e-12)
    assert T[0] == pytest.approx(0.05 ** 3, rel=1e-12)


def test_projection_against_camera_matrix():
    """Projected means equal K p / p_z with K = [[fx, 0, cx], [0, -fy, cy], [0, 0, 1]]."""
    rng = np.random.default_rng(2)
    ang = rng.uniform(0, 2 * np.pi)
    R = np.array([[math.cos(ang), 0, -math.sin(ang)], [0, 1, 0], [math.sin(ang), 0, math.cos(ang)]])
    cam = orr.camera(R, [0.3, -0.2, -5.0], W, H, 0.5)
    means = rng.uniform(-1, 1, (20, 3))
    _, m2, _, valid = orr.project(means, np.full((20, 3), 0.1), [[1, 0, 0, 0]] * 20, cam)
    K = np.array([[cam["fx"], 0, cam["cx"]], [0, -cam["fy"], cam["cy"]], [0, 0, 1.0]])
    h = (K @ (R @ (means - cam["centre"]).T)).T
    np.testing.assert_allclose(m2[valid], (h[:, :2] / h[:, 2:])[valid], rtol=1e-12)


def test_ewa_covariance_against_numerical_jacobian():
    rng = np.random.default_rng(3)
    cam = _cam(centre=(0.2, 0.1, -3.0))
    n = 15
    means, scales, quats, _, _ = _scene(n, 3)
    _, m2, s2, _ = orr.project(means, scales, quats, cam)
    Rq = orr.quat_rotation(quats)

    def proj(pt):
        p = cam["rot"] @ (pt - cam["centre"])
        return np.array([cam["cx"] + cam["fx"] * p[0] / p[2], cam["cy"] - cam["fy"] * p[1] / p[2]])

    for k in range(n):
        Jn = np.zeros((2, 3))
        for c in range(3):
            e = np.zeros(3)
            e[c] = 1e-6
            Jn[:, c] = (proj(means[k] + e) - proj(means[k] - e)) / 2e-6
        S3 = Rq[k] @ np.diag(scales[k] ** 2) @ Rq[k].T
        np.testing.assert_allclose(s2[k], Jn @ S3 @ Jn.T + orr.LOWPASS * np.eye(2), rtol=1e-7, atol=1e-9)


def test_footprint_bound_holds_every_contributing_pixel():
    cam = _cam()
    means, scales, quats, op, _ = _scene(40, 4, big=True)
    _, m2, s2, valid = orr.project(means, scales, quats, cam)
    r = orr.footprint_radius(s2, op)
    jj, ii = np.mgrid[0:H, 0:W]
    for k in range(40):
        if not valid[k]:
            continue
        d = np.stack([ii + 0.5 - m2[k, 0], jj + 0.5 - m2[k, 1]], axis=-1)
        q = np.einsum("...i,ij,...j->...", d, np.linalg.inv(s2[k]), d)
        a = op[k] * np.exp(-0.5 * q)
        inside = (np.abs(d[..., 0]) <= r[k]) & (np.abs(d[..., 1]) <= r[k])
        assert np.all(inside[a >= orr.ALPHA_MIN])
        if r[k] < 0:
            assert not np.any(a >= orr.ALPHA_MIN)


def test_backward_against_finite_differences():
    W2, H2 = 14, 10
    cam2 = orr.camera(np.eye(3), (0, 0, -4.0), W2, H2, 0.15)
    means, scales, quats, op, col = _scene(25, 5, spread=0.5, big=True)
    rng = np.random.default_rng(6)
    g = rng.normal(size=(H2, W2, 3))
    g_c, g_o = orr.render_backward(means, scales, quats, op, col, cam2, W2, H2, g)

    def loss(o, c):
        img, _ = orr.render(means, scales, quats, o, c, cam2, W2, H2)
        return float(np.sum(img * g))

    _, _, margin = orr.render(means, scales, quats, op, col, cam2, W2, H2, with_margin=True)
    assert margin.min() > 1e-5            # no decision sits on a threshold at this draw
    for k in range(25):
        for c in range(3):
            cp, cm = col.copy(), col.copy()
            cp[k, c] += 1e-3
            cm[k, c] -= 1e-3
            assert (loss(op, cp) - loss(op, cm)) / 2e-3 == pytest.approx(g_c[k, c], rel=1e-9, abs=1e-12)
        h = 1e-7
        opp, opm = op.copy(), op.copy()
        opp[k] += h
        opm[k] -= h
        fd = (loss(opp, col) - loss(opm, col)) / (2 * h)
        assert fd == pytest.approx(g_o[k], rel=1e-5, abs=1e-7)
    assert np.abs(g_c).sum() > 0 and np.abs(g_o).sum() > 0
