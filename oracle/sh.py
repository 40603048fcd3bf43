"""FP64 CPU oracle for real spherical harmonics (the comparison appearance model).

TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the benchmark's
CPU-baseline leg; never by the product path. Shares no code with the CUDA path.

Sec. 3.2 (Background, Spherical Harmonics) writes the appearance as
f(d; c) = sum_{l<=L} sum_{m=-l..l} c_lm Y_l^m(d). The paper does not fix the
real-SH convention; this oracle uses the orthonormal real basis built from the
associated Legendre functions with the Condon-Shortley phase:

    Y_lm = sqrt(2) K_lm P_l^m(cos t) cos(m p)        m > 0
    Y_l0 = K_l0 P_l(cos t)
    Y_lm = sqrt(2) K_l|m| P_l^|m|(cos t) sin(|m| p)  m < 0
    K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)

with (t, p) the polar and azimuthal angles of d and coefficient index l^2+l+m.
P_l^m is evaluated by the standard three-term recurrence in l from P_m^m.
No +0.5 offset and no clamp are applied (the Sec. 3.2 equation has none).
"""
from __future__ import annotations

import math

import numpy as np


def _legendre_table(x, degree):
    """P_l^m(x) (with Condon-Shortley phase) and dP_l^m/dx for 0 <= m <= l <= degree."""
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P = {}
    for m in range(degree + 1):
        # P_m^m = (-1)^m (2m-1)!! (1-x^2)^{m/2}
        dfact = 1.0
        for j in range(1, 2 * m, 2):
            dfact *= j
        P[(m, m)] = ((-1.0) ** m) * dfact * s ** m
        if m + 1 <= degree:
            P[(m + 1, m)] = x * (2 * m + 1) * P[(m, m)]
        for l in range(m + 2, degree + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    dP = {}
    for (l, m), val in P.items():
        # (x^2 - 1) dP_l^m/dx = l x P_l^m - (l + m) P_{l-1}^m
        prev = P.get((l - 1, m), np.zeros_like(x))
        dP[(l, m)] = (l * x * val - (l + m) * prev) / (x * x - 1.0)
    return P, dP


def _norm(l, m):
    return math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))


def basis(d, degree=3, need_grad=False):
    """Real SH basis values (N, (degree+1)^2) at unit directions d (N, 3).

    With need_grad, also returns the surface gradient (N, nb, 3) of each basis
    function on the sphere (tangent to the sphere at d).
    """
    d = np.asarray(d, dtype=np.float64)
    x = np.clip(d[:, 2], -1.0, 1.0)
    t = np.arccos(x)
    ph = np.arctan2(d[:, 1], d[:, 0])
    P, dP = _legendre_table(x, degree)
    nb = (degree + 1) ** 2
    Y = np.zeros((d.shape[0], nb))
    dY_dt = np.zeros_like(Y)
    dY_dp = np.zeros_like(Y)
    sin_t = np.sin(t)
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = _norm(l, am)
            pl = P[(l, am)]
            dpl_dt = dP[(l, am)] * (-sin_t)        # d/dt P(cos t)
            if m > 0:
                trig, dtrig = math.sqrt(2.0) * np.cos(m * ph), -math.sqrt(2.0) * m * np.sin(m * ph)
            elif m < 0:
                trig, dtrig = math.sqrt(2.0) * np.sin(am * ph), math.sqrt(2.0) * am * np.cos(am * ph)
            else:
                trig, dtrig = np.ones_like(ph), np.zeros_like(ph)
            j = l * l + l + m
            Y[:, j] = K * pl * trig
            dY_dt[:, j] = K * dpl_dt * trig
            dY_dp[:, j] = K * pl * dtrig
    if not need_grad:
        return Y
    e_t = np.stack([np.cos(t) * np.cos(ph), np.cos(t) * np.sin(ph), -np.sin(t)], axis=-1)
    e_p = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=-1)
    grad = dY_dt[..., None] * e_t[:, None, :] + (dY_dp / sin_t[:, None])[..., None] * e_p[:, None, :]
    return Y, grad


def _dirs(means, cam):
    r = np.asarray(means, dtype=np.float64) - np.asarray(cam, dtype=np.float64)[None, :]
    dist = np.sqrt(np.sum(r * r, axis=-1))
    return r / dist[:, None], dist


def forward(coeffs, means, cam, degree=3):
    """rgb_i,c = sum_j coeffs[j, c, i] Y_j(d_i); coeffs [(degree+1)^2][3][N] -> (N, 3) float64."""
    d, _ = _dirs(means, cam)
    Y = basis(d, degree)
    return np.einsum("jcn,nj->nc", np.asarray(coeffs, dtype=np.float64), Y)


def backward(coeffs, means, cam, g_rgb, degree=3):
    """(g_coeffs [(degree+1)^2][3][N], g_means (N, 3)) for the upstream g_rgb (N, 3)."""
    d, dist = _dirs(means, cam)
    Y, gY = basis(d, degree, need_grad=True)
    g = np.asarray(g_rgb, dtype=np.float64)
    C = np.asarray(coeffs, dtype=np.float64)
    g_coeffs = np.einsum("nc,nj->jcn", g, Y)
    w = np.einsum("jcn,nc->nj", C, g)                 # dL/dY_j
    g_d = np.einsum("nj,njk->nk", w, gY)              # tangent gradient on the sphere
    g_d = g_d - np.sum(g_d * d, axis=-1, keepdims=True) * d
    return g_coeffs, g_d / dist[:, None]
