"""Pins of the FP64 NASGabor oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails at least one of them:
  * special cases that reduce to textbook / library functions (SG, von Mises-Fisher),
  * the Sec. 5.1 closed-form integral where it is exact, by quadrature,
  * the unit mass of the approximately normalised kernel at k = 0,
  * the special values at d = +-z,
  * invariance under a joint rotation and under x -> -x (evenness in d.x),
  * the Supp. C cosine frame against a library rotation,
  * every analytic derivative against central finite differences in FP64.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.stats import vonmises_fisher

from oracle import nasgabor as ng
from paper_2606_09794_gb300 import inputs
from tests._quadrature import integrate_lobe

RNG = np.random.default_rng(20260)


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _random_frames(n, rng):
    q = _unit(rng.standard_normal((n, 4)))
    return (q,) + ng.frame_from_quat(q)


# ---------------------------------------------------------------------------
# Special cases
# ---------------------------------------------------------------------------

def test_isotropic_no_carrier_is_spherical_gaussian():
    """a = 0, k = 0: G reduces to the normalised SG of the distributions table,
    lam/(2 pi (1 - e^{-2 lam})) exp(lam (z.d - 1))."""
    n = 2000
    d = _unit(RNG.standard_normal((n, 3)))
    _, x, z = _random_frames(n, RNG)
    lam = np.exp(RNG.uniform(-2, 5, n))
    G = ng.lobe(d, x, z, lam, np.zeros(n), np.zeros(n), ng.NORM_APPROX)
    u = np.sum(d * z, -1)
    sg = lam / (2 * np.pi * (1 - np.exp(-2 * lam))) * np.exp(lam * (u - 1))
    np.testing.assert_allclose(G, sg, rtol=1e-12, atol=0)


def test_isotropic_no_carrier_is_von_mises_fisher_density():
    """a = 0, k = 0, normalised: the von Mises-Fisher density with concentration lam (scipy)."""
    for lam in (0.5, 3.0, 40.0):
        z = _unit(RNG.standard_normal(3))
        q = Rotation.align_vectors([z], [[0, 0, 1]])[0].as_quat()  # x, y, z, w
        qw = np.array([q[3], q[0], q[1], q[2]])
        x_ax, z_ax = ng.frame_from_quat(qw[None, :])
        np.testing.assert_allclose(z_ax[0], z, atol=1e-12)
        d = _unit(RNG.standard_normal((500, 3)))
        n = d.shape[0]
        G = ng.lobe(d, np.broadcast_to(x_ax, d.shape), np.broadcast_to(z_ax, d.shape),
                    np.full(n, lam), np.zeros(n), np.zeros(n), ng.NORM_APPROX)
        ref = vonmises_fisher(z, lam).pdf(d)
        np.testing.assert_allclose(G, ref, rtol=1e-10)


def test_isotropic_with_carrier_is_sg_times_carrier():
    """a = 0: tau = 0, E = 1 and G = SG(d) (1 + cos(k d.x))/2; checks the carrier's argument is d.x."""
    n = 1000
    d = _unit(RNG.standard_normal((n, 3)))
    _, x, z = _random_frames(n, RNG)
    lam = np.exp(RNG.uniform(0, 4, n))
    k = RNG.uniform(0, 40, n)
    G = ng.lobe(d, x, z, lam, np.zeros(n), k, ng.NORM_NONE)
    u, v = np.sum(d * z, -1), np.sum(d * x, -1)
    np.testing.assert_allclose(G, np.exp(lam * (u - 1)) * np.cos(k * v / 2) ** 2, rtol=1e-12, atol=1e-300)


def test_special_values_at_poles():
    """Sec. 5.1: G(z) = 1 and G(-z) = 0 for the unnormalised kernel; C^-1 at z when normalised."""
    n = 50
    _, x, z = _random_frames(n, RNG)
    lam = np.exp(RNG.uniform(0, 6, n))
    a = RNG.uniform(0, 2, n)
    k = RNG.uniform(0, 40, n)
    # random frames: z.z is 1 only up to rounding, so the values are the limits
    np.testing.assert_allclose(ng.lobe(z, x, z, lam, a, k, ng.NORM_NONE), 1.0, rtol=1e-12)
    # (at -z the limit depends on the path: along d.x = 0 it is e^{-2 lam}, not the
    # convention G(-z) = 0, so only the exact antipode is checked below)
    np.testing.assert_allclose(ng.lobe(z, x, z, lam, a, k, ng.NORM_APPROX), ng.norm_approx(lam, a), rtol=1e-12)
    # exact world-axis frame: the Sec. 5.1 special values hold exactly
    e = np.array([[0.0, 0.0, 1.0]])
    xe = np.array([[1.0, 0.0, 0.0]])
    one = np.ones(1)
    assert ng.lobe(e, xe, e, 7 * one, 0.4 * one, 3 * one, ng.NORM_NONE)[0] == 1.0
    assert ng.lobe(-e, xe, e, 7 * one, 0.4 * one, 3 * one, ng.NORM_NONE)[0] == 0.0
    # exact poles along the world axis: q = identity, d = +-e_z, all finite
    G, par = ng.lobe(e, xe, e, np.array([5.0]), np.array([0.3]), np.array([2.0]), ng.NORM_APPROX, True)
    assert np.isfinite(G).all() and all(np.isfinite(v).all() for v in par.values())
    G, par = ng.lobe(-e, xe, e, np.array([5.0]), np.array([0.3]), np.array([2.0]), ng.NORM_APPROX, True)
    assert G[0] == 0.0 and all((v == 0).all() for v in par.values())


def test_near_pole_is_continuous():
    """Directions 1e-3 .. 1e-7 rad from +z approach the pole value C^-1 h(0) = C^-1."""
    lam, a, k = 20.0, 0.7, 3.0
    vals = []
    for eps in (1e-3, 1e-5, 1e-7):
        d = np.array([[math.sin(eps), 0.0, math.cos(eps)]])
        vals.append(ng.lobe(d, np.array([[1.0, 0, 0]]), np.array([[0, 0, 1.0]]), np.array([lam]),
                            np.array([a]), np.array([k]), ng.NORM_APPROX)[0])
    lim = ng.norm_approx(lam, a)
    errs = [abs(v - lim) / lim for v in vals]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-10


# ---------------------------------------------------------------------------
# Integrals (Sec. 5.1 closed form; NASG normalisation of the distributions table)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lam,a", [(0.3, 0.0), (1.0, 0.5), (4.0, 1.5), (60.0, 0.9), (900.0, 0.3)])
def test_approx_normalised_kernel_has_unit_mass_without_carrier(lam, a):
    """k = 0: int C^-1 p E d omega = 1 (the NASG constant is exact)."""
    val = integrate_lobe(ng.lobe, lam, a, 0.0, ng.NORM_APPROX)
    assert abs(val - 1.0) < 1e-9


@pytest.mark.parametrize("lam,a,k", [
    (0.3, 0.0, 3.0), (1.0, 0.0, 2.0), (2.5, 0.0, 40.0), (7.0, 0.0, 7.0), (30.0, 0.0, 12.0),
    (1.0, 0.5, 0.0), (3.0, 1.2, 0.0), (200.0, 0.7, 0.0),
])
def test_closed_form_integral_where_exact(lam, a, k):
    """Sec. 5.1 closed form vs quadrature of the unnormalised kernel, for a = 0 or k = 0.

    Covers Lambda > k, Lambda < k (sinhc continued to sin x / x) and Lambda = k."""
    quad = integrate_lobe(ng.lobe, lam, a, k, ng.NORM_NONE)
    closed = float(ng.integral_closed_form(lam, a, k))
    assert abs(quad - closed) <= 1e-9 * abs(closed)


def test_closed_form_integral_is_approximate_for_anisotropic_carrier():
    """For a > 0 and k > 0 the printed closed form departs from the quadrature
    (reading recorded in the design notes); the deviation is small but real."""
    quad = integrate_lobe(ng.lobe, 1.0, 0.5, 2.0, ng.NORM_NONE)
    closed = float(ng.integral_closed_form(1.0, 0.5, 2.0))
    rel = abs(quad - closed) / quad
    assert 1e-3 < rel < 0.1


@pytest.mark.parametrize("lam,k", [(3.0, 9.0), (500.0, 9.0), (800.0, 40.0), (40.0, 40.0)])
def test_exact_normalisation_has_unit_mass_where_closed_form_exact(lam, k):
    """a = 0: the exactly normalised lobe integrates to 1, also at lam where
    sinh(Lambda) overflows FP64 and at k = Lambda."""
    val = integrate_lobe(ng.lobe, lam, 0.0, k, ng.NORM_EXACT)
    assert abs(val - 1.0) < 1e-9


@pytest.mark.parametrize("big", [1e-3, 0.7, 5.0, 300.0, 710.0, 2000.0])
@pytest.mark.parametrize("k", [0.0, 0.3, 2.0, 8.0, 40.0])
def test_exp_sinhc_against_arbitrary_precision(big, k):
    """e^{-Lambda} sinhc(sqrt(Lambda^2 - k^2)) against mpmath at 50 digits, across
    the sinh / sin / series branches and past FP64's sinh overflow."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    L, K = mpmath.mpf(big), mpmath.mpf(k)
    sig = L * L - K * K
    if sig > 0:
        s = mpmath.sqrt(sig)
        ref = mpmath.exp(-L) * mpmath.sinh(s) / s
    elif sig < 0:
        t = mpmath.sqrt(-sig)
        ref = mpmath.exp(-L) * mpmath.sin(t) / t
    else:
        ref = mpmath.exp(-L)
    got = float(ng._exp_sinhc(np.float64(big), np.float64(k)))
    assert abs(got - float(ref)) <= 1e-13 * abs(float(ref)) + 1e-300


@pytest.mark.parametrize("lam,a", [(0.05, 0.2), (1.0, 0.5), (700.0, 1.0), (1000.0, 0.0)])
def test_closed_form_without_carrier_is_the_nasg_mass(lam, a):
    """k = 0: Psi = 1, so the closed form is the NASG constant's reciprocal
    2 pi (1 - e^{-2 lam}) / (lam sqrt(1+a)), at every Lambda."""
    nasg = 2.0 * math.pi * -math.expm1(-2.0 * lam) / (lam * math.sqrt(1.0 + a))
    assert abs(float(ng.integral_closed_form(lam, a, 0.0)) - nasg) <= 1e-13 * nasg


@pytest.mark.parametrize("lam,a,k", [(0.8, 0.3, 1.3), (2.0, 0.5, 3.0), (600.0, 0.7, 6.0), (3.0, 0.0, 3.0),
                                     (0.4, 0.2, 30.0)])
def test_exact_normalisation_partials_against_finite_differences(lam, a, k):
    """Complex-step partials of 1/int G against central differences of the real closed form."""
    got = ng._exact_norm_partials(np.array(lam), np.array(a), np.array(k))
    base = (lam, a, k)
    for j in range(3):
        h = 1e-6 * max(1.0, abs(base[j]))
        hi = list(base)
        lo = list(base)
        hi[j] += h
        lo[j] -= h
        fd = (1.0 / ng.integral_closed_form(*hi) - 1.0 / ng.integral_closed_form(*lo)) / (2.0 * h)
        assert abs(float(got[j]) - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(1.0 / ng.integral_closed_form(*base)))


# ---------------------------------------------------------------------------
# Invariances
# ---------------------------------------------------------------------------

def _quat_mul(p, q):
    w1, x1, y1, z1 = (p[..., i] for i in range(4))
    w2, x2, y2, z2 = (q[..., i] for i in range(4))
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=-1)


def test_joint_rotation_invariance():
    n = 3000
    q, x, z = _random_frames(n, RNG)
    d = _unit(RNG.standard_normal((n, 3)))
    lam, a, k = np.exp(RNG.uniform(0, 5, n)), RNG.uniform(0, 1, n), RNG.uniform(0, 8, n)
    G0 = ng.lobe(d, x, z, lam, a, k)
    r = _unit(RNG.standard_normal(4))
    R = Rotation.from_quat([r[1], r[2], r[3], r[0]]).as_matrix()
    x2, z2 = ng.frame_from_quat(_quat_mul(np.broadcast_to(r, q.shape), q))
    np.testing.assert_allclose(x2, x @ R.T, atol=1e-14)
    G1 = ng.lobe(d @ R.T, x2, z2, lam, a, k)
    np.testing.assert_allclose(G1, G0, rtol=1e-11, atol=1e-300)


def test_even_in_d_dot_x():
    """Rotating the frame by pi about z (x -> -x, y -> -y) leaves G unchanged."""
    n = 2000
    q, x, z = _random_frames(n, RNG)
    d = _unit(RNG.standard_normal((n, 3)))
    lam, a, k = np.exp(RNG.uniform(0, 5, n)), RNG.uniform(0, 1, n), RNG.uniform(0, 8, n)
    q2 = _quat_mul(q, np.broadcast_to(np.array([0.0, 0, 0, 1]), q.shape))
    x2, z2 = ng.frame_from_quat(q2)
    np.testing.assert_allclose(x2, -x, atol=1e-14)
    np.testing.assert_allclose(z2, z, atol=1e-14)
    np.testing.assert_allclose(ng.lobe(d, x2, z2, lam, a, k), ng.lobe(d, x, z, lam, a, k), rtol=1e-9)


def test_anisotropy_orientation():
    """With a > 0 the lobe is narrower along x than along y: G(tilt toward x) < G(tilt toward y)."""
    x = np.array([[1.0, 0, 0]])
    z = np.array([[0, 0, 1.0]])
    t = 0.2
    dx = np.array([[math.sin(t), 0, math.cos(t)]])
    dy = np.array([[0, math.sin(t), math.cos(t)]])
    args = (np.array([10.0]), np.array([1.0]), np.array([0.0]))
    assert ng.lobe(dx, x, z, *args) < ng.lobe(dy, x, z, *args)


def test_quat_frame_matches_library_rotation():
    q = _unit(RNG.standard_normal((200, 4)))
    x, z = ng.frame_from_quat(q)
    R = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], -1)).as_matrix()
    np.testing.assert_allclose(x, R[:, :, 0], atol=1e-14)
    np.testing.assert_allclose(z, R[:, :, 2], atol=1e-14)


def test_cos_frame_is_a_rotation_and_agrees_with_quat_mode():
    """Supp. C frame: orthonormal with y = z x x, and the same G as the QUAT frame of that rotation."""
    n = 500
    ang = RNG.uniform(0.05, np.pi - 0.05, (n, 3))
    c = np.cos(ang)
    x, z = ng.frame_from_cos(c)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=-1)
    np.testing.assert_allclose(R @ np.swapaxes(R, -1, -2), np.broadcast_to(np.eye(3), R.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-13)
    qs = Rotation.from_matrix(R).as_quat()
    q = np.stack([qs[:, 3], qs[:, 0], qs[:, 1], qs[:, 2]], -1)
    xq, zq = ng.frame_from_quat(q)
    np.testing.assert_allclose(xq, x, atol=1e-13)
    np.testing.assert_allclose(zq, z, atol=1e-13)


def test_parameter_count_matches_paper_table():
    """Efficiency table: NASGabor with 1/2/4 lobes has 12/21/39 appearance parameters
    (3 diffuse + 9 per lobe in the Supp. C parameterisation); SH degree 3 has 48.
    The storage column is consistent with those counts at one primitive count."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "efficiency_table.json")) as f:
        tab = json.load(f)
    for row in tab["nasgabor"]:
        assert 3 + ng.lobe_planes(ng.FRAME_COS) * row["lobes"] == row["params"]
    assert (3 + 1) ** 2 * 3 == tab["sh3"]["params"]
    # storage deltas per extra FP32 parameter give one primitive count
    rows = {r["lobes"]: r for r in tab["nasgabor"]}
    per_param = []
    for a, b in ((1, 2), (2, 4)):
        dp = rows[b]["params"] - rows[a]["params"]
        per_param.append((rows[b]["storage_mb"] - rows[a]["storage_mb"]) / dp)
    dp = tab["sh3"]["params"] - rows[1]["params"]
    per_param.append((tab["sh3"]["storage_mb"] - rows[1]["storage_mb"]) / dp)
    assert max(per_param) / min(per_param) < 1.001


# ---------------------------------------------------------------------------
# Derivatives (Supp. E/F, readings R3-R8) against central finite differences
# ---------------------------------------------------------------------------

def _fd_case(frame_mode, act_mode, n, n_lobes, seed, lam_hi=50.0):
    rng = np.random.default_rng(seed)
    P = ng.lobe_planes(frame_mode)
    if act_mode == ng.ACT_RAW:
        w = inputs.point_cloud_workload(n, n_lobes, seed, frame_mode)
        params = w.params.astype(np.float64)
        base = 4 if frame_mode == ng.FRAME_QUAT else 3
        params[base] = np.log(np.exp(rng.uniform(0, math.log(lam_hi), n * n_lobes)))
        # spread k over the paper's full [0, 40] range, and w over [-1, 1]
        params[base + 2] = np.arctanh(rng.uniform(0.01, 39.9, n * n_lobes) / 20 - 1)
        params[base + 3:base + 6] = np.arctanh(rng.uniform(-0.95, 0.95, (3, n * n_lobes)))
        c0, means, cam = w.c0, w.means, w.cam
    else:
        params = np.zeros((P, n * n_lobes))
        if frame_mode == ng.FRAME_QUAT:
            params[0:4] = rng.standard_normal((4, n * n_lobes))
        else:
            params[0:3] = np.cos(rng.uniform(0.1, np.pi - 0.1, (3, n * n_lobes)))
        base = 4 if frame_mode == ng.FRAME_QUAT else 3
        params[base] = rng.uniform(0.5, lam_hi, n * n_lobes)
        params[base + 1] = rng.uniform(0.0, 2.0, n * n_lobes)
        params[base + 2] = rng.uniform(0.0, 40.0, n * n_lobes)
        params[base + 3:base + 6] = rng.uniform(-1, 1, (3, n * n_lobes))
        c0 = rng.uniform(0, 1, (3, n))
        means = rng.uniform(0, 1, (n, 3))
        cam = np.array([0.0, 0.0, 3.0])
    g_rgb = rng.standard_normal((n, 3))
    return params, c0, means, cam, g_rgb


def _assert_fd(an, fd, where, rtol=2e-6, atol_frac=1e-8):
    """|analytic - FD| <= rtol |FD| + atol_frac max|FD| (the FD noise floor is ~1e-10 absolute)."""
    tol = rtol * np.abs(fd) + atol_frac * np.max(np.abs(fd)) + 1e-14
    bad = np.abs(an - fd) > tol
    assert not bad.any(), (where, an[bad][:4], fd[bad][:4])


def _per_prim_loss(params, c0, means, cam, g_rgb, n_lobes, fm, nm, am, var=ng.VAR_NASGABOR):
    return np.sum(g_rgb * ng.forward(params, c0, means, cam, n_lobes, fm, nm, am, var), axis=-1)


@pytest.mark.parametrize("frame_mode,variant", [(ng.FRAME_QUAT, ng.VAR_NASGABOR), (ng.FRAME_COS, ng.VAR_NASGABOR),
                                                (ng.FRAME_QUAT, ng.VAR_NASG), (ng.FRAME_QUAT, ng.VAR_SG),
                                                (ng.FRAME_QUAT, ng.VAR_PHASE), (ng.FRAME_COS, ng.VAR_PHASE)])
@pytest.mark.parametrize("norm_mode", [ng.NORM_APPROX, ng.NORM_NONE, ng.NORM_EXACT])
@pytest.mark.parametrize("act_mode", [ng.ACT_RAW, ng.ACT_IDENTITY])
def test_backward_matches_central_differences(frame_mode, variant, norm_mode, act_mode):
    n, L = 64, 3
    params, c0, means, cam, g_rgb = _fd_case(frame_mode, act_mode, n, L, seed=11)
    phase = np.random.default_rng(5).uniform(0.0, 2.0 * np.pi, n * L)
    params = inputs.variant_planes(params, phase, frame_mode, variant)
    g_p, g_c0, g_mu = ng.backward(params, c0, means, cam, g_rgb, L, frame_mode, norm_mode, act_mode, variant)
    args = (L, frame_mode, norm_mode, act_mode, variant)
    P = params.shape[0]
    for p in range(P):
        for l in range(L):
            idx = np.arange(n) * L + l
            h = 1e-6 * np.maximum(1.0, np.abs(params[p, idx]))
            pp, pm = params.copy(), params.copy()
            pp[p, idx] += h
            pm[p, idx] -= h
            fd = (_per_prim_loss(pp, c0, means, cam, g_rgb, *args)
                  - _per_prim_loss(pm, c0, means, cam, g_rgb, *args)) / (2 * h)
            an = g_p[p, idx]
            _assert_fd(an, fd, (p, l))
    for c in range(3):
        h = 1e-6
        mp, mm = means.astype(np.float64).copy(), means.astype(np.float64).copy()
        mp[:, c] += h
        mm[:, c] -= h
        fd = (_per_prim_loss(params, c0, mp, cam, g_rgb, *args)
              - _per_prim_loss(params, c0, mm, cam, g_rgb, *args)) / (2 * h)
        _assert_fd(g_mu[:, c], fd, c)
    np.testing.assert_array_equal(g_c0, g_rgb.T)


def test_normalisation_lambda_derivative_sign():
    """Reading R4: dC^-1/dlam at lam = 0.7, a = 0.4 is 0.13542 (finite differences);
    the printed '+' numerator would give 0.36449."""
    lam, a, h = 0.7, 0.4, 1e-6
    fd = (ng.norm_approx(lam + h, a) - ng.norm_approx(lam - h, a)) / (2 * h)
    d = np.array([[0.0, 0.0, 1.0]])
    _, par = ng.lobe(d, np.array([[1.0, 0, 0]]), d, np.array([lam]), np.array([a]), np.array([0.0]),
                     ng.NORM_APPROX, True)
    # at d = z (pole, tau := 0, h = 1) dG/dlam = dC^-1/dlam
    assert abs(par["lam"][0] - fd) < 1e-8
    assert abs(fd - 0.13542) < 1e-5
    em = math.exp(-2 * lam)
    printed = (math.sqrt(1 + a) * (1 - em) + 2 * lam * math.sqrt(1 + a) * em) / (2 * math.pi * (1 - em) ** 2)
    assert abs(printed - 0.36449) < 1e-5


def test_sharp_lobe_derivatives():
    """Derivatives stay consistent with finite differences at sharpness up to 1e3."""
    n, L = 32, 2
    params, c0, means, cam, g_rgb = _fd_case(ng.FRAME_QUAT, ng.ACT_IDENTITY, n, L, seed=5, lam_hi=1000.0)
    args = (L, ng.FRAME_QUAT, ng.NORM_APPROX, ng.ACT_IDENTITY)
    # aim lobe 0 of every primitive close to its view direction so that G is not negligible
    d, _ = ng.view_directions(means, cam)
    for i in range(n):
        zt = d[i] + 0.01 * np.random.default_rng(i).standard_normal(3)
        zt /= np.linalg.norm(zt)
        q = Rotation.align_vectors([zt], [[0, 0, 1]])[0].as_quat()
        params[0:4, i * L] = [q[3], q[0], q[1], q[2]]
    g_p = ng.backward(params, c0, means, cam, g_rgb, *args)[0]
    assert np.isfinite(g_p).all()
    for p in range(10):
        idx = np.arange(n) * L
        # the naive FP64 lobe carries ~2 lam 1e-16 relative noise, so the step is not tiny
        h = 1e-5 * np.maximum(np.abs(params[p, idx]), 1e-2)
        pp, pm = params.copy(), params.copy()
        pp[p, idx] += h
        pm[p, idx] -= h
        fd = (_per_prim_loss(pp, c0, means, cam, g_rgb, *args) - _per_prim_loss(pm, c0, means, cam, g_rgb, *args)) / (2 * h)
        _assert_fd(g_p[p, idx], fd, p, rtol=1e-5, atol_frac=1e-7)


# ---------------------------------------------------------------------------
# Lobe families (NASG, SG, phase-shifted carrier)
# ---------------------------------------------------------------------------

def test_sg_family_is_the_von_mises_fisher_density():
    """SG (a = 0, k = 0) normalised: exactly the von Mises-Fisher density with
    concentration lam about z (scipy), per lobe through the whole forward."""
    w = inputs.variant_workload(200, 2, 31, "sg", activated=True)
    rgb = ng.forward(w.params, w.c0, w.means, w.cam, 2, act_mode=ng.ACT_IDENTITY, variant=ng.VAR_SG)
    d, _ = ng.view_directions(w.means, w.cam)
    _, z = ng.frame_from_quat(np.moveaxis(w.params[0:4].reshape(4, 200, 2), 0, -1).astype(np.float64))
    lam = w.params[4].reshape(200, 2).astype(np.float64)
    ref = w.c0.T.astype(np.float64).copy()
    for i in range(200):
        for j in range(2):
            dens = vonmises_fisher(z[i, j], lam[i, j]).pdf(d[i])
            ref[i] += w.params[5:8, 2 * i + j].astype(np.float64) * dens
    np.testing.assert_allclose(rgb, ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("variant", [ng.VAR_NASG, ng.VAR_SG])
def test_families_equal_nasgabor_with_fixed_parameters(variant):
    """NASG and SG are the NASGabor lobe at k = 0 (and a = 0): same colours and
    the same gradients for every stored plane (identity activations)."""
    n, L = 50, 3
    w = inputs.point_cloud_workload(n, L, 32, activated=True)
    full = w.params.astype(np.float64).copy()
    full[6] = 0.0
    if variant == ng.VAR_SG:
        full[5] = 0.0
    fam = inputs.variant_planes(full, None, "quat", variant)
    for norm in (ng.NORM_APPROX, ng.NORM_EXACT):
        a = ng.forward(full, w.c0, w.means, w.cam, L, norm_mode=norm, act_mode=ng.ACT_IDENTITY)
        b = ng.forward(fam, w.c0, w.means, w.cam, L, norm_mode=norm, act_mode=ng.ACT_IDENTITY, variant=variant)
        np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-13)
        ga = ng.backward(full, w.c0, w.means, w.cam, w.g_rgb, L, norm_mode=norm, act_mode=ng.ACT_IDENTITY)[0]
        gb = ng.backward(fam, w.c0, w.means, w.cam, w.g_rgb, L, norm_mode=norm, act_mode=ng.ACT_IDENTITY,
                         variant=variant)[0]
        keep = [0, 1, 2, 3, 4] + ([5] if variant == ng.VAR_NASG else []) + [7, 8, 9]
        np.testing.assert_allclose(gb, ga[keep], rtol=1e-10, atol=1e-12)


def test_phase_carrier_at_zero_phase_is_nasgabor():
    n, L = 40, 2
    w = inputs.point_cloud_workload(n, L, 33)
    ph = inputs.variant_planes(w.params.astype(np.float64), np.zeros(n * L), "quat", "phase")
    for norm in (ng.NORM_APPROX, ng.NORM_EXACT, ng.NORM_NONE):
        np.testing.assert_allclose(ng.forward(ph, w.c0, w.means, w.cam, L, norm_mode=norm, variant=ng.VAR_PHASE),
                                   ng.forward(w.params, w.c0, w.means, w.cam, L, norm_mode=norm),
                                   rtol=1e-13, atol=1e-13)


def test_phase_carrier_reflection_symmetry():
    """Reflecting d across the plane normal to x flips v = d.x and leaves u: the
    phase family obeys G(d; phi) = G(reflected d; -phi)."""
    rng = np.random.default_rng(34)
    n = 300
    q = _unit(rng.standard_normal((n, 4)))
    x, z = ng.frame_from_quat(q)
    d = _unit(rng.standard_normal((n, 3)))
    dr = d - 2.0 * np.sum(d * x, axis=-1, keepdims=True) * x
    lam, a, k = rng.uniform(0.5, 30, n), rng.uniform(0, 1, n), rng.uniform(0, 40, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    g1 = ng.lobe(d, x, z, lam, a, k, ng.NORM_APPROX, phi=phi)
    g2 = ng.lobe(dr, x, z, lam, a, k, ng.NORM_APPROX, phi=-phi)
    np.testing.assert_allclose(g1, g2, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("lam,k,phi", [(3.0, 9.0, 0.7), (40.0, 12.0, 2.0), (5.0, 5.0, math.pi), (200.0, 30.0, 4.0)])
def test_phase_carrier_exact_normalisation_has_unit_mass(lam, k, phi):
    """a = 0: with the cos(phi)-scaled closed form (the sin part integrates to 0)
    the exactly normalised phase-shifted lobe integrates to 1."""
    val = integrate_lobe(lambda *args, **kw: ng.lobe(*args, **kw, phi=np.full(np.shape(args[3]), phi)),
                         lam, 0.0, k, ng.NORM_EXACT)
    assert abs(val - 1.0) < 1e-9


def _lobe_mp(u, v, lam, a, k, s2):
    """The Sec. 5.1 / Supp. F lobe written out in mpmath from its definition
    (kappa = (1+u)/2, tau = a v^2/(1-u^2), E = kappa^tau, p = e^{2 lam (E kappa - 1)},
    h = (1 + cos(k v))/2, approximate C^-1), with 1 - u^2 = s2 supplied."""
    import mpmath as mp
    kappa = (1 + u) / 2
    tau = a * v * v / s2
    E = kappa ** tau
    p = mp.exp(2 * lam * (E * kappa - 1))
    h = (1 + mp.cos(k * v)) / 2
    cinv = lam * mp.sqrt(1 + a) / (2 * mp.pi * (1 - mp.exp(-2 * lam)))
    return cinv * p * E * h


@pytest.mark.parametrize("theta", [1e-2, 1e-5, 1e-7, 1e-9, 1e-12])
@pytest.mark.parametrize("side", [1.0, -1.0])
def test_lobe_near_poles_matches_50_digit_definition(theta, side):
    """Directions theta from +z (side +1) and -z (side -1), down to 1e-12 rad: the FP64
    lobe value and its partials (u, v, lam, a, k) against the definition evaluated in
    50-digit arithmetic at the normalised direction, partials by mpmath.diff. The
    FP64 forms 1 - u u and (1 + u)/2 would lose ~1 % at 1e-7 rad and all digits below
    ~1e-8 rad."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for lam, a, k, psi in ((1.0, 0.5, 3.0, 0.3), (30.0, 0.8, 7.0, 1.1), (1000.0, 0.3, 2.0, 0.0)):
        d = np.array([math.sin(theta) * math.cos(psi), math.sin(theta) * math.sin(psi), side * math.cos(theta)])
        x = np.array([1.0, 0.0, 0.0])
        z = np.array([0.0, 0.0, 1.0])
        G, par = ng.lobe(d[None], x[None], z[None], np.array([lam]), np.array([a]), np.array([k]), need_grad=True)
        dm = [mp.mpf(float(c)) for c in d]
        nrm = mp.sqrt(sum(c * c for c in dm))
        dm = [c / nrm for c in dm]
        u0, v0 = dm[2], dm[0]
        s2 = dm[0] ** 2 + dm[1] ** 2

        def f(u, v, lm, aa, kk, s2_=None):
            return _lobe_mp(u, v, lm, aa, kk, (1 - u) * (1 + u) if s2_ is None else s2_)

        L_, A_, K_ = mp.mpf(lam), mp.mpf(a), mp.mpf(k)
        ref = f(u0, v0, L_, A_, K_, s2)
        dnorm = float(np.dot(d, d))
        got = {"G": float(G[0]), "u": float(np.dot(par["z"][0], d)) / dnorm, "v": float(np.dot(par["x"][0], d)) / dnorm,
               "lam": float(par["lam"][0]), "a": float(par["a"][0]), "k": float(par["k"][0])}
        # derivative in u at fixed v: 1 - u^2 varies with u; at the base point it equals s2
        want = {"G": ref,
                "u": mp.diff(lambda t: f(t, v0, L_, A_, K_), u0),
                "v": mp.diff(lambda t: f(u0, t, L_, A_, K_, s2), v0),
                "lam": mp.diff(lambda t: f(u0, v0, t, A_, K_, s2), L_),
                "a": mp.diff(lambda t: f(u0, v0, L_, t, K_, s2), A_),
                "k": mp.diff(lambda t: f(u0, v0, L_, A_, t, s2), K_)}
        for key, w in want.items():
            w = float(w)
            assert abs(got[key] - w) <= 1e-9 * abs(w) + 1e-300, (theta, side, lam, key, got[key], w)
