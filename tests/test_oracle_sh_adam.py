"""Pins of the FP64 SH and optimiser oracles.

SH: orthonormality on a quadrature grid exact to degree 6, Y_00, the addition
theorem (band energy (2l+1)/(4 pi) at every direction), agreement with scipy's
complex spherical harmonics, and central finite differences of the backward.
Adam: agreement with torch.optim.Adam in float64; the fused step's masking; the
fitting step's zero-loss fixed point and its gradient against finite differences.
"""
import math

import numpy as np
import pytest
import torch
from scipy.special import sph_harm_y

from oracle import adam as oad
from oracle import nasgabor as ng
from oracle import sh as osh
from paper_2606_09794_gb300 import inputs

RNG = np.random.default_rng(777)


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def test_sh_orthonormal_gram():
    # Gauss-Legendre in cos(t) with 8 nodes x 16 uniform phi: exact for degree <= 6 products
    xg, wg = np.polynomial.legendre.leggauss(8)
    ph = np.arange(16) * 2 * np.pi / 16
    X, PH = np.meshgrid(xg, ph, indexing="ij")
    W = (wg[:, None] * np.full(16, 2 * np.pi / 16)[None, :]).reshape(-1)
    s = np.sqrt(1 - X ** 2)
    d = np.stack([s * np.cos(PH), s * np.sin(PH), X], -1).reshape(-1, 3)
    Y = osh.basis(d, 3)
    gram = (Y * W[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-13)


def test_sh_constant_and_addition_theorem():
    d = _unit(RNG.standard_normal((400, 3)))
    Y = osh.basis(d, 3)
    np.testing.assert_allclose(Y[:, 0], 1 / (2 * math.sqrt(math.pi)), rtol=1e-15)
    for l in range(4):
        band = Y[:, l * l:(l + 1) ** 2]
        np.testing.assert_allclose(np.sum(band ** 2, -1), (2 * l + 1) / (4 * math.pi), rtol=1e-12)


def test_sh_matches_scipy_complex_harmonics():
    """Real basis from scipy's complex Y_l^m (Condon-Shortley phase included):
    sqrt(2) Re Y_l^m for m > 0, Y_l^0, sqrt(2) Im Y_l^|m| for m < 0."""
    d = _unit(RNG.standard_normal((300, 3)))
    t = np.arccos(d[:, 2])
    ph = np.arctan2(d[:, 1], d[:, 0])
    Y = osh.basis(d, 3)
    for l in range(4):
        for m in range(-l, l + 1):
            c = sph_harm_y(l, abs(m), t, ph)
            ref = c.real if m == 0 else math.sqrt(2) * (c.real if m > 0 else c.imag)
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-13)


def test_sh_backward_matches_central_differences():
    n = 200
    means = RNG.uniform(0, 1, (n, 3))
    cam = np.array([0.0, 0.0, 3.0])
    coeffs = 0.3 * RNG.standard_normal((16, 3, n))
    g = RNG.standard_normal((n, 3))
    gc, gm = osh.backward(coeffs, means, cam, g)
    np.testing.assert_allclose(gc, np.einsum("nc,nj->jcn", g, osh.basis(ng.view_directions(means, cam)[0])))
    for c in range(3):
        h = 1e-6
        mp, mm = means.copy(), means.copy()
        mp[:, c] += h
        mm[:, c] -= h
        fd = (np.sum(g * osh.forward(coeffs, mp, cam), -1) - np.sum(g * osh.forward(coeffs, mm, cam), -1)) / (2 * h)
        np.testing.assert_allclose(gm[:, c], fd, rtol=1e-6, atol=1e-9)


def test_adam_matches_torch_in_float64():
    theta0 = RNG.standard_normal(64)
    th = theta0.copy()
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    p = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8, foreach=False)
    for t in range(1, 11):
        g = RNG.standard_normal(64) * (10.0 ** RNG.uniform(-6, 2, 64))
        th, m, v = oad.adam_update(th, m, v, g, t, lr=3e-3)
        opt.zero_grad()
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=0, atol=1e-15)


def test_bf16_round_matches_torch():
    x = (RNG.standard_normal(10000) * 10.0 ** RNG.uniform(-5, 5, 10000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oad.bf16_round(x), ref)
    np.testing.assert_array_equal(inputs.quantize_bf16(x).astype(np.float64), ref)


def test_fused_step_updates_only_visible():
    n, L = 64, 4
    w = inputs.point_cloud_workload(n, L, 3)
    P = w.params.shape[0]
    zeros = np.zeros((P, n * L))
    idx = np.arange(0, n, 3)
    out = oad.fused_step(w.params, zeros, zeros, w.c0, np.zeros((3, n)), np.zeros((3, n)), w.means, w.cam,
                         w.g_rgb, idx, L, t=1)
    hidden = np.setdiff1d(np.arange(n), idx)
    lobe_hidden = (hidden[:, None] * L + np.arange(L)).reshape(-1)
    np.testing.assert_array_equal(out["master"][:, lobe_hidden], w.params[:, lobe_hidden])
    np.testing.assert_array_equal(out["m"][:, lobe_hidden], 0.0)
    # first Adam step: m = (1 - b1) g and the gradient is the oracle backward at the BF16 values
    lobe_vis = (idx[:, None] * L + np.arange(L)).reshape(-1)
    pq = oad.bf16_round(w.params[:, lobe_vis])
    c0q = oad.bf16_round(w.c0[:, idx])
    g_p, g_c0, _ = ng.backward(pq, c0q, w.means[idx], w.cam, w.g_rgb[idx], L)
    np.testing.assert_allclose(out["m"][:, lobe_vis], 0.1 * g_p, rtol=1e-12)
    np.testing.assert_allclose(out["c0_m"][:, idx], 0.1 * g_c0, rtol=1e-12)
    np.testing.assert_allclose(out["rgb"], ng.forward(pq, c0q, w.means[idx], w.cam, L), rtol=1e-15)


def test_fused_step_mse_gradient_matches_finite_differences():
    """loss "mse": the gradient the step uses (m / (1 - b1) after a cold first step) is
    the derivative of the mean over listed primitives and channels of the squared colour
    error, by central differences of the oracle's forward at the BF16 values."""
    n, L = 12, 3
    w = inputs.point_cloud_workload(n, L, 41)
    P = w.params.shape[0]
    idx = np.array([1, 2, 5, 7, 11])
    master = oad.bf16_round(w.params)          # on the BF16 grid, so FD moves it freely
    target = np.random.default_rng(42).uniform(0, 2, (n, 3))
    zeros = np.zeros((P, n * L))
    out = oad.fused_step(master, zeros, zeros, w.c0, np.zeros((3, n)), np.zeros((3, n)), w.means, w.cam, target,
                         idx, L, t=1, loss="mse")
    g = out["m"] / 0.1
    lobes = (idx[:, None] * L + np.arange(L)).reshape(-1)
    c0q = oad.bf16_round(w.c0[:, idx])

    def loss_at(p):
        col = ng.forward(p[:, lobes], c0q, w.means[idx], w.cam, L)
        return np.sum((col - target[idx]) ** 2) / (3 * len(idx))

    assert abs(loss_at(master) - out["loss"]) <= 1e-15 * out["loss"]
    rng = np.random.default_rng(43)
    for p in range(P):
        for j in rng.choice(lobes, 4, replace=False):
            h = 1e-6 * max(1.0, abs(master[p, j]))
            pp, pm = master.copy(), master.copy()
            pp[p, j] += h
            pm[p, j] -= h
            fd = (loss_at(pp) - loss_at(pm)) / (2 * h)
            tol = 1e-6 * abs(fd) + 64 * np.finfo(float).eps * out["loss"] / h + 1e-14
            assert abs(g[p, j] - fd) <= tol, (p, j, g[p, j], fd)
    # c0: d loss / d c0_ic = 2 (c_ic - t_ic) / (3 n_listed)
    np.testing.assert_allclose(out["c0_m"][:, idx] / 0.1, (2.0 * (out["rgb"] - target[idx]) / (3 * len(idx))).T,
                               rtol=1e-12)


def test_fused_step_mse_at_own_colours_does_not_move():
    """A target equal to the model's own colours gives a zero gradient: from a cold state
    nothing moves (m = v = 0, and the update 0 / (0 + eps) is 0)."""
    n, L = 32, 4
    w = inputs.point_cloud_workload(n, L, 44)
    P = w.params.shape[0]
    idx = np.arange(0, n, 2)
    zeros = np.zeros((P, n * L))
    lobes = (idx[:, None] * L + np.arange(L)).reshape(-1)
    own = np.zeros((n, 3))
    own[idx] = ng.forward(oad.bf16_round(w.params[:, lobes]), oad.bf16_round(w.c0[:, idx]), w.means[idx], w.cam, L)
    out = oad.fused_step(w.params, zeros, zeros, w.c0, np.zeros((3, n)), np.zeros((3, n)), w.means, w.cam, own,
                         idx, L, t=1, loss="mse")
    assert out["loss"] == 0.0
    np.testing.assert_array_equal(out["master"], w.params.astype(np.float64))
    np.testing.assert_array_equal(out["c0"], w.c0.astype(np.float64))


def _bf16_exact(x):
    return oad.bf16_round(x)


def test_fit_step_fixed_point_at_teacher():
    """A student equal to the teacher (padded with zero-weight lobes) has zero loss and does not move."""
    n, Lt, Ls = 40, 4, 16
    t = inputs.point_cloud_workload(n, Lt, 21)
    teacher = _bf16_exact(t.params)
    t_c0 = _bf16_exact(t.c0)
    P = teacher.shape[0]
    student = np.zeros((P, n * Ls))
    student[0] = 1.0  # identity quaternions for the padding lobes
    tv = teacher.reshape(P, n, Lt)
    sv = student.reshape(P, n, Ls)
    sv[:, :, :Lt] = tv
    student = sv.reshape(P, -1)
    dirs = inputs.fit_directions(0, 5, 64)
    zeros = np.zeros_like(student)
    new, mse = oad.fit_step(student, zeros, zeros, t_c0, np.zeros((3, n)), np.zeros((3, n)), teacher, t_c0,
                            dirs, Ls, Lt, t=1)
    # zero up to the summation order of the two mixtures: residuals ~1e-14 give
    # gradients ~1e-11 at lam ~ 1e3, which Adam's eps turns into steps below
    # lr * 1e-11 / eps = 1e-6, against lr = 1e-3 for any real gradient
    assert mse < 1e-24
    np.testing.assert_allclose(new["student"], student, rtol=0, atol=1e-5)
    np.testing.assert_allclose(new["c0"], t_c0, rtol=0, atol=1e-5)


def test_fit_step_gradient_matches_finite_differences():
    n, Lt, Ls = 6, 2, 3
    tw = inputs.point_cloud_workload(n, Lt, 31)
    sw = inputs.point_cloud_workload(n, Ls, 32)
    dirs = inputs.fit_directions(1, 9, 8)
    P = sw.params.shape[0]
    zeros = np.zeros((P, n * Ls))
    st = sw.params.astype(np.float64)
    new, _ = oad.fit_step(st, zeros, zeros, sw.c0, np.zeros((3, n)), np.zeros((3, n)),
                          tw.params, tw.c0, dirs, Ls, Lt, t=1, bf16_storage=False)
    g = new["m"] / 0.1
    target = oad.field_colours(tw.params, tw.c0, dirs, Lt)

    def per_prim_loss(p):
        col = oad.field_colours(p, sw.c0, dirs, Ls)
        return np.mean((col - target) ** 2, axis=(1, 2))

    for p in range(P):
        for l in range(Ls):
            idx = np.arange(n) * Ls + l
            h = 1e-6 * np.maximum(1.0, np.abs(st[p, idx]))
            pp, pm = st.copy(), st.copy()
            pp[p, idx] += h
            pm[p, idx] -= h
            fd = (per_prim_loss(pp) - per_prim_loss(pm)) / (2 * h)
            # noise floor of the difference quotient: a few ulps of the loss over 2h
            tol = 2e-6 * np.abs(fd) + 64 * np.finfo(float).eps * per_prim_loss(st) / h + 1e-14
            assert (np.abs(g[p, idx] - fd) <= tol).all(), (p, l)
