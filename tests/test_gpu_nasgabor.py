"""GPU parity of the NASGabor kernels (through the C ABI) against the FP64 oracle.

Colours: |c_gpu - c_oracle| <= 1e-5 + 4 nu per output (nu = oracle sensitivity
floor, tests/_parity.py), for FP32 parameters and for BF16 parameters alike (the
oracle is fed the dequantised values; the arithmetic is FP32 in both).
Gradients: relative L2 error <= 1e-4 per parameter plane, for c0 and for the
means, and element by element (grad_report): |dg| <= 1e-4 |g| + 4 nu + f +
1e-12 max|g of the plane|, f the FP32 rounding floor of the gradients that are
sums of terms of opposite sign (_chain_floor).
"""
import math

import numpy as np
import pytest

from oracle import nasgabor as ong
from paper_2606_09794_gb300 import inputs
from tests._parity import chain_floor as _chain_floor
from tests._parity import colour_report, grad_report, rel_l2, sensitivity_floor

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4
COLOUR_BASE = 1e-5


def _dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t if dtype is None else t.to(dtype)


def _prepare(w, bf16):
    """Device tensors and the float32 values the kernel reads (dequantised for BF16)."""
    import torch
    if bf16:
        pq = inputs.quantize_bf16(w.params)
        cq = inputs.quantize_bf16(w.c0)
        return (_dev(w.params).to(torch.bfloat16), _dev(w.c0).to(torch.bfloat16), pq, cq)
    return _dev(w.params), _dev(w.c0), w.params, w.c0


def _check_forward(lib, w, bf16, norm="approx", act="raw", base=None, family="nasgabor"):
    import torch
    params, c0, p_np, c0_np = _prepare(w, bf16)
    means = _dev(w.means)
    rgb = lib.nasgabor_eval_fwd(params, c0, means, w.cam, w.n_lobes, w.frame_mode, norm, act, family=family)
    torch.cuda.synchronize()
    gpu = rgb.cpu().numpy()
    assert np.isfinite(gpu).all()

    def fwd(p, c, m, cam):
        return ong.forward(p, c, m, cam, w.n_lobes, w.frame_mode, norm, act, family)

    ref, nu = sensitivity_floor(fwd, (p_np, c0_np, w.means, w.cam), (0, 1, 2, 3))
    rep = colour_report(gpu, ref, nu, base if base is not None else COLOUR_BASE)
    assert rep["violations"] == 0, rep
    return rep


def _check_backward(lib, w, bf16, norm="approx", act="raw", family="nasgabor"):
    import torch
    params, c0, p_np, c0_np = _prepare(w, bf16)
    means = _dev(w.means)
    g_rgb = _dev(w.g_rgb)
    g_p, g_c0, g_mu = lib.nasgabor_eval_bwd(params, means, w.cam, g_rgb, w.n_lobes, w.frame_mode, norm, act,
                                            family=family)
    torch.cuda.synchronize()
    r_p, r_c0, r_mu = ong.backward(p_np, c0_np, w.means, w.cam, w.g_rgb, w.n_lobes, w.frame_mode, norm, act,
                                   family)
    g_p = g_p.cpu().numpy()
    assert np.isfinite(g_p).all()
    errs = [rel_l2(g_p[p], r_p[p]) for p in range(g_p.shape[0])]
    assert max(errs) <= GRAD_TOL, errs
    np.testing.assert_array_equal(g_c0.cpu().numpy(), w.g_rgb.T)
    assert rel_l2(g_mu.cpu().numpy(), r_mu) <= GRAD_TOL
    # element by element: |dg| <= 1e-4 |g| + 4 nu + the projection floor + 1e-12 max|g of the plane|
    P, n, L = g_p.shape[0], w.n, w.n_lobes

    def bwd(p_, c_, m_, cm_):
        gp_, _, gm_ = ong.backward(p_, c_, m_, cm_, w.g_rgb, L, w.frame_mode, norm, act, family)
        return np.concatenate([gp_.ravel(), gm_.ravel()])

    ref, nu = sensitivity_floor(bwd, (p_np, c0_np, w.means, w.cam), (0, 1, 2, 3))
    groups = np.concatenate([np.repeat(np.arange(P), n * L), np.full(3 * n, P)])
    scale = np.array([np.abs(ref[groups == g]).max() for g in range(P + 1)])
    floor = _chain_floor(p_np, w.means, w.cam, w.g_rgb, L, w.frame_mode, norm, act, family)
    got = np.concatenate([g_p.ravel(), g_mu.cpu().numpy().ravel()])
    rep = grad_report(got, ref, nu, atol=1e-12 * scale[groups] + floor)
    assert rep["violations"] == 0, rep
    return errs


CASES = [
    # frame, N, L, bf16, norm, act, seed
    ("quat", 4096, 4, False, "approx", "raw", 1001),   # the small parity workload
    ("quat", 1037, 8, False, "approx", "raw", 7),      # ragged tail, 4-lobe vector path
    ("quat", 777, 3, False, "approx", "raw", 8),       # scalar path (L % 4 != 0)
    ("quat", 301, 1, False, "approx", "raw", 9),
    ("cos", 1029, 4, False, "approx", "raw", 10),
    ("cos", 555, 5, False, "approx", "raw", 11),
    ("quat", 600, 4, False, "none", "raw", 12),
    ("quat", 513, 5, False, "approx", "identity", 13),
    ("cos", 700, 4, False, "approx", "identity", 14),
    ("quat", 4096, 8, True, "approx", "raw", 15),
    ("cos", 999, 4, True, "approx", "raw", 16),
    ("quat", 333, 3, True, "approx", "raw", 17),
    ("quat", 1037, 8, False, "exact", "raw", 18),     # Sec. 5.1 exact normalisation
    ("cos", 555, 5, False, "exact", "raw", 19),
    ("quat", 513, 4, False, "exact", "identity", 20),
    ("quat", 4096, 8, True, "exact", "raw", 22),       # staged path, run-time flags
]


def _exact_branch_workload():
    """Identity-mode lobes whose (lam, a, k) cover every branch of the exact
    normalisation: Lam = lam (1 + a) equal to k, |Lam^2 - k^2| on both sides of 1,
    Lam << k (sin branch), Lam >> k up to 2e3 (rearranged derivative), tiny Lam."""
    lam = [0.05, 0.3, 1.0, 2.0, 3.0, 3.0, 7.9, 8.0, 12.0, 30.0, 100.0, 1000.0, 1000.0, 0.45, 20.0, 39.0]
    a = [0.0, 0.2, 0.5, 0.0, 0.0, 1.0, 0.01, 0.0, 0.5, 0.3, 1.0, 1.0, 0.0, 0.1, 1.0, 0.0]
    k = [0.1, 30.0, 1.5, 2.1, 3.0, 5.9, 8.0, 8.2, 0.0, 40.0, 8.0, 40.0, 0.5, 0.4, 39.9, 39.0]
    n, L = 3 * len(lam), 2                       # every triple appears in 6 lobes
    w = inputs.point_cloud_workload(n, L, 23, "quat", activated=True)
    for row, vals in ((4, lam), (5, a), (6, k)):
        w.params[row] = np.tile(np.asarray(vals, dtype=np.float32), n * L // len(lam))
    return w


FAMILY_CASES = [
    # family, N, L, bf16, norm, act, seed
    ("nasg", 1037, 8, False, "approx", "raw", 41),
    ("nasg", 4096, 8, True, "approx", "raw", 42),      # staged path
    ("sg", 777, 3, False, "approx", "raw", 43),
    ("sg", 4096, 4, True, "approx", "raw", 44),
    ("phase", 1029, 6, False, "approx", "raw", 45),
    ("phase", 4096, 8, True, "exact", "raw", 46),
    ("phase", 513, 5, False, "exact", "identity", 47),
    ("nasg", 300, 2, False, "exact", "identity", 48),
    ("phase", 2048, 4, False, "none", "raw", 49),
]


@pytest.mark.parametrize("family,n,L,bf16,norm,act,seed", FAMILY_CASES)
def test_lobe_family_parity(lib, family, n, L, bf16, norm, act, seed):
    """NASG, SG and the phase-shifted carrier against the oracle's families."""
    w = inputs.variant_workload(n, L, seed, family, activated=(act == "identity"))
    _check_forward(lib, w, bf16, norm, act, family=family)
    _check_backward(lib, w, bf16, norm, act, family=family)


@pytest.mark.parametrize("family", ["nasg", "sg", "phase"])
def test_lobe_family_fused_equals_separate_passes(lib, family):
    import torch
    w = inputs.variant_workload(2048, 8, 50, family)
    params, c0 = _dev(w.params).to(torch.bfloat16), _dev(w.c0).to(torch.bfloat16)
    means, g_rgb = _dev(w.means), _dev(w.g_rgb)
    rgb = lib.nasgabor_eval_fwd(params, c0, means, w.cam, 8, family=family)
    g = lib.nasgabor_eval_bwd(params, means, w.cam, g_rgb, 8, family=family)
    f = lib.nasgabor_fused_fwd_bwd(params, c0, means, w.cam, g_rgb, 8, family=family)
    torch.cuda.synchronize()
    torch.testing.assert_close(f[0], rgb, rtol=1e-6, atol=1e-6)
    fg, sg = f[1].cpu().numpy(), g[0].cpu().numpy()
    assert max(rel_l2(fg[p], sg[p]) for p in range(fg.shape[0])) < 1e-6


def test_lobe_family_rejections(lib):
    import torch
    w = inputs.variant_workload(64, 4, 51, "sg")
    params, c0, means = _dev(w.params), _dev(w.c0), _dev(w.means)
    with pytest.raises(ValueError):  # planes of the wrong family
        lib.nasgabor_eval_fwd(params, c0, means, w.cam, 4, family="phase")
    with pytest.raises(ValueError):  # families take QUAT frames
        lib.nasgabor_eval_fwd(params, c0, means, w.cam, 4, frame_mode="cos", family="sg")
    st = lib.TrainState(_dev(inputs.point_cloud_workload(64, 4, 52).params), c0.clone())
    with pytest.raises(lib.NasgError):
        lib.nasgabor_fused_step(st, means, w.cam, torch.zeros((64, 3), device="cuda"), 4, 1, family="sg")


def _phase_cancellation_workload():
    """Identity-mode phase-carrier lobes where the exactly normalised lobe's integral
    nearly vanishes: phi at or next to pi and k << Lam = lam (1 + a), where
    1 + cos(phi) Psi reaches ~1e-6 (both branches of its cancellation-free form:
    sig > 1 and small Lam)."""
    import itertools
    combos = list(itertools.product([0.2, 0.6, 3.0, 50.0, 700.0], [0.0, 0.5, 0.94], [1e-3, 0.06, 0.5],
                                    [math.pi, math.pi - 1e-3, 3.140625]))
    L = 4
    n = (len(combos) + L - 1) // L
    w = inputs.variant_workload(n, L, 53, "phase", activated=True)
    vals = np.array(combos * 2, dtype=np.float32)[: n * L]
    for j, row in enumerate((4, 5, 6, 7)):      # lam, a, k, phi after the 4 quaternion planes
        w.params[row] = vals[:, j]
    return w


def test_phase_exact_normalisation_near_zero_integral(lib):
    """Colours with the usual bound; gradients element by element with the oracle's
    sensitivity floor (here the carrier argument k v + phi ~ pi carries k v to a few
    digits only, in the inputs themselves, so a plain relative bound would grade the
    FP32 representation of phi rather than the kernel) and the projection floor. The
    carrier is formed by angle addition from phi/2 and k v/2: the rounded sum k v + phi
    alone would put ~1e-4 relative error into it here (h ~ 1e-7 at phi = pi - 1e-3)."""
    import torch
    w = _phase_cancellation_workload()
    _check_forward(lib, w, False, "exact", "identity", family="phase")
    L, n = w.n_lobes, w.n
    g_p, _, g_mu = lib.nasgabor_eval_bwd(_dev(w.params), _dev(w.means), w.cam, _dev(w.g_rgb), L, "quat", "exact",
                                         "identity", family="phase")
    torch.cuda.synchronize()

    def bwd(p_, c_, m_, cm_):
        gp_, _, gm_ = ong.backward(p_, c_, m_, cm_, w.g_rgb, L, "quat", "exact", "identity", "phase")
        return np.concatenate([gp_.ravel(), gm_.ravel()])

    ref, nu = sensitivity_floor(bwd, (w.params, w.c0, w.means, w.cam), (0, 1, 2, 3), draws=8)
    got = np.concatenate([g_p.cpu().numpy().ravel(), g_mu.cpu().numpy().ravel()])
    floor = _chain_floor(w.params, w.means, w.cam, w.g_rgb, L, "quat", "exact", "identity", "phase")
    rep = grad_report(got, ref, nu, atol=1e-12 * np.abs(ref).max() + floor)
    assert rep["finite"] and rep["violations"] == 0, rep


def test_exact_normalisation_branches(lib):
    w = _exact_branch_workload()
    _check_forward(lib, w, False, "exact", "identity")
    _check_backward(lib, w, False, "exact", "identity")


@pytest.mark.parametrize("frame,n,L,bf16,norm,act,seed", CASES)
def test_forward_parity(lib, frame, n, L, bf16, norm, act, seed):
    w = inputs.point_cloud_workload(n, L, seed, frame, activated=(act == "identity"))
    _check_forward(lib, w, bf16, norm, act)


@pytest.mark.parametrize("frame,n,L,bf16,norm,act,seed", CASES)
def test_backward_parity(lib, frame, n, L, bf16, norm, act, seed):
    w = inputs.point_cloud_workload(n, L, seed, frame, activated=(act == "identity"))
    _check_backward(lib, w, bf16, norm, act)


@pytest.mark.parametrize("bf16", [False, True])
def test_fused_equals_separate_passes(lib, bf16):
    import torch
    w = inputs.point_cloud_workload(2049, 8, 21)
    params, c0, _, _ = _prepare(w, bf16)
    means, g_rgb = _dev(w.means), _dev(w.g_rgb)
    rgb = lib.nasgabor_eval_fwd(params, c0, means, w.cam, 8)
    g = lib.nasgabor_eval_bwd(params, means, w.cam, g_rgb, 8)
    f = lib.nasgabor_fused_fwd_bwd(params, c0, means, w.cam, g_rgb, 8)
    torch.cuda.synchronize()
    # same arithmetic, separately compiled: rounding may differ in ill-conditioned entries
    torch.testing.assert_close(f[0], rgb, rtol=1e-6, atol=1e-6)
    fg = f[1].cpu().numpy()
    sg = g[0].cpu().numpy()
    assert max(rel_l2(fg[p], sg[p]) for p in range(fg.shape[0])) < 1e-6
    torch.testing.assert_close(f[2], g[1], rtol=0, atol=0)
    # the fused pass reduce-scatters dLoss/dd over the slice (another summation order),
    # and dLoss/dmu projects out the radial part (cancellation): a looser bound
    assert rel_l2(f[3].cpu().numpy(), g[2].cpu().numpy()) < 1e-5


def test_index_list_and_accumulate(lib):
    import torch
    w = inputs.point_cloud_workload(1000, 4, 22)
    params, c0 = _dev(w.params), _dev(w.c0)
    means, g_rgb = _dev(w.means), _dev(w.g_rgb)
    full = lib.nasgabor_eval_fwd(params, c0, means, w.cam, 4)
    idx_np = np.sort(np.random.default_rng(3).choice(1000, 317, replace=False)).astype(np.int32)
    idx = _dev(idx_np)
    rgb = torch.full((1000, 3), -7.0, device="cuda")
    lib.nasgabor_eval_fwd(params, c0, means, w.cam, 4, idx=idx, rgb=rgb)
    gpu = rgb.cpu().numpy()
    assert (gpu[np.setdiff1d(np.arange(1000), idx_np)] == -7.0).all()
    np.testing.assert_array_equal(gpu[idx_np], full.cpu().numpy()[idx_np])
    # backward with an index list touches only the listed primitives; accumulate adds
    g1 = lib.nasgabor_eval_bwd(params, means, w.cam, g_rgb, 4)
    gp = torch.zeros_like(g1[0])
    gc = torch.zeros_like(g1[1])
    gm = torch.zeros_like(g1[2])
    lib.nasgabor_eval_bwd(params, means, w.cam, g_rgb, 4, idx=idx, g_params=gp, g_c0=gc, g_means=gm)
    lib.nasgabor_eval_bwd(params, means, w.cam, g_rgb, 4, idx=idx, g_params=gp, g_c0=gc, g_means=gm,
                          accumulate=True)
    torch.cuda.synchronize()
    lobes = (idx_np[:, None] * 4 + np.arange(4)).reshape(-1)
    np.testing.assert_allclose(gp.cpu().numpy()[:, lobes], 2 * g1[0].cpu().numpy()[:, lobes], rtol=1e-6)
    others = np.setdiff1d(np.arange(4000), lobes)
    assert (gp.cpu().numpy()[:, others] == 0).all()
    np.testing.assert_allclose(gm.cpu().numpy()[idx_np], 2 * g1[2].cpu().numpy()[idx_np], rtol=1e-6)


def _axis_pole_workload():
    """Frames with exact axes (q = (0, 1, 0, 0): z = -e_z, x = e_x; q = (1, 0, 0, 0): z = e_z),
    a camera on the z axis and centres at 0, 1e-3, 1e-5 and 1e-7 rad from it, offset along
    x, y or both: FP32 holds these directions to full relative accuracy, so the lobe sees
    the intended angle. Lobe 0 of each primitive faces the view direction (u -> +1), lobe 1
    faces away (u -> -1); sharpness 1, 30 and 1e3."""
    cam = np.array([0.0, 0.0, 3.0], dtype=np.float32)
    angles, lams, offs = [0.0, 1e-3, 1e-5, 1e-7], [1.0, 30.0, 1000.0], [(1.0, 0.0), (0.0, 1.0), (0.6, 0.8)]
    rows = [(e, lam, o) for e in angles for lam in lams for o in offs]
    n, L = len(rows), 2
    means = np.array([[2 * math.sin(e) * o[0], 2 * math.sin(e) * o[1], 3.0 - 2 * math.cos(e)] for e, _, o in rows],
                     np.float32)
    p = np.zeros((10, n * L), np.float32)
    p[1, 0::2] = 1.0
    p[0, 1::2] = 1.0
    p[4] = np.repeat(np.log([r[1] for r in rows]), L).astype(np.float32)
    p[5] = math.log(0.6)
    p[6] = math.atanh(3.0 / 20 - 1)
    p[7:10] = math.atanh(0.5)
    c0 = np.full((3, n), 0.25, np.float32)
    g_rgb = np.random.default_rng(5).standard_normal((n, 3)).astype(np.float32)
    return inputs.Workload(n, L, "quat", p, c0, means, cam, g_rgb, None)


@pytest.mark.parametrize("bf16", [False, True])
def test_poles_and_near_poles(lib, bf16):
    """Exact +-z view directions and directions 1e-3, 1e-5, 1e-7 rad from the axis on frames
    with exact axes (the values are exact in BF16 too): colours within the usual bound, the
    exact-pole colour in closed form, zero gradients at the exact anti-pole, and every
    gradient element (parameter planes and means, fused pass and separate backward) within
    1e-4 |g| + 4 nu + 1e-12 max|g of the plane| of the oracle, plus for the means the FP32
    rounding floor of their projection (_chain_floor; the frame axes here are exact, so the
    frame planes get none)."""
    import torch
    w = _axis_pole_workload()
    dt = torch.bfloat16 if bf16 else torch.float32
    n, L = w.n, w.n_lobes
    rep = _check_forward(lib, w, bf16)
    gpu = lib.nasgabor_eval_fwd(_dev(w.params).to(dt), _dev(w.c0).to(dt), _dev(w.means), w.cam, L).cpu().numpy()
    pq = inputs.quantize_bf16(w.params) if bf16 else w.params
    for i in range(3):   # exact pole, lam = 1, 30, 1e3 (lobe 1, at the anti-pole, adds 0): c0 + w C^-1
        lam, a, wt = (math.exp(float(pq[4, 6 * i])), math.exp(float(pq[5, 6 * i])), math.tanh(float(pq[7, 6 * i])))
        cinv = lam * math.sqrt(1 + a) / (2 * math.pi * (1 - math.exp(-2 * lam)))
        np.testing.assert_allclose(gpu[3 * i], 0.25 + wt * cinv, rtol=1e-5)
    g_p, g_c0, g_mu = lib.nasgabor_eval_bwd(_dev(w.params).to(dt), _dev(w.means), w.cam, _dev(w.g_rgb), L)
    f = lib.nasgabor_fused_fwd_bwd(_dev(w.params).to(dt), _dev(w.c0).to(dt), _dev(w.means), w.cam, _dev(w.g_rgb), L)
    torch.cuda.synchronize()
    assert (g_p.cpu().numpy()[:, 1:18:2] == 0).all()  # exact anti-pole (first 9 primitives): zero gradients

    def bwd(p_, c_, m_, cm_):
        gp_, _, gm_ = ong.backward(p_, c_, m_, cm_, w.g_rgb, L)
        return np.concatenate([gp_.ravel(), gm_.ravel()])

    ref, nu = sensitivity_floor(bwd, (pq, w.c0, w.means, w.cam), (0, 1, 2, 3), draws=8)
    groups = np.concatenate([np.repeat(np.arange(10), n * L), np.full(3 * n, 10)])
    scale = np.array([np.abs(ref[groups == g]).max() for g in range(11)])
    floor = _chain_floor(pq, w.means, w.cam, w.g_rgb, L, frame_planes=False)   # exact axes: no frame rounding
    assert np.isfinite(floor).all()
    for name, gp, gm in (("bwd", g_p, g_mu), ("fused", f[1], f[3])):
        got = np.concatenate([gp.cpu().numpy().ravel(), gm.cpu().numpy().ravel()])
        r = grad_report(got, ref, nu, atol=1e-12 * scale[groups] + floor)
        assert r["finite"] and r["violations"] == 0, (name, r)
    assert rep["violations"] == 0


NEAR_POLE_ANGLES = [0.0, 1e-3, 1e-5, 1e-7]
NEAR_POLE_LAMS = [1.0, 30.0, 1000.0]


def _near_pole_workload(frame, bf16, seed, L=8):
    """One primitive per (angle, lam, side, offset direction): its view direction is at
    the given angle from +z (or -z) of one of its lobes (lobe index i mod L, sharpness
    lam), offset towards that lobe's x, y or (x + y)/sqrt(2) (tau = a, 0, a/2 in the
    limit); the other lobes are random. Frames from random quaternions (QUAT) or raw
    cosines (COS); the direction is placed against the frame of the stored (for BF16:
    dequantised) values, then rounded to FP32 means, so the oracle sees the inputs the
    GPU reads."""
    spec = [(e, lam, sgn, off) for e in NEAR_POLE_ANGLES for lam in NEAR_POLE_LAMS for sgn in (1.0, -1.0)
            for off in ("x", "y", "xy")]
    n = len(spec)
    w = inputs.point_cloud_workload(n, L, seed, frame)
    base = 4 if frame == "quat" else 3
    p = w.params.copy()
    lobe_of = np.arange(n) % L
    for i, (_, lam, _, _) in enumerate(spec):
        p[base, i * L + lobe_of[i]] = math.log(lam)
    if bf16:
        p = inputs.quantize_bf16(p)
    act = ong.activate(ong.split_planes(p, n, L, frame), frame)
    x, z = ong._frames(act, frame)
    means = np.zeros((n, 3))
    for i, (e, _, sgn, off) in enumerate(spec):
        zz, xx = z[i, lobe_of[i]], x[i, lobe_of[i]]
        yy = np.cross(zz, xx)
        t = {"x": xx, "y": yy, "xy": (xx + yy) / math.sqrt(2.0)}[off]
        means[i] = 2.0 * sgn * (math.cos(e) * zz + math.sin(e) * t)
    c0 = inputs.quantize_bf16(w.c0) if bf16 else w.c0
    return inputs.Workload(n, L, frame, p.astype(np.float32), c0, means.astype(np.float32),
                           np.zeros(3, np.float32), w.g_rgb, None)


@pytest.mark.parametrize("frame,bf16", [("quat", False), ("quat", True), ("cos", False), ("cos", True)])
def test_near_pole_gradients_elementwise(lib, frame, bf16):
    """The pole edge cases on frames of any orientation: view directions at
    0, 1e-3, 1e-5 and 1e-7 rad from +-z of a lobe with sharpness 1, 30 and 1e3, in the fused
    pass (the launch the benchmark times), the separate backward and the register path (a
    misaligned view). At 1e-3 and 1e-5 rad every gradient element of every plane and of the
    means is compared with the oracle, |dg| <= 1e-4 |g| + 4 nu + 1e-12 max|g of the plane|
    + the projection floor f, nu the oracle's own change when every FP32 input moves by
    8 ulps (the GPU forms d and the frame axes in a few FP32 roundings each; at 1e-5 rad
    the gradients move by ~1e-3..1e-2 of themselves under such moves) and f the FP32
    rounding floor of the frame-plane and means gradients (_chain_floor: near the anti-pole
    dLoss/dd is ~1e7 and almost radial, its tangential part ~1). At 0 and 1e-7 rad an FP32 direction and an FP32
    frame of arbitrary orientation cannot be placed that close (their components carry
    ~1e-7 absolute rounding), so the gradients there are only required finite; frames with
    exact axes, where FP32 does resolve 1e-7 rad, are compared element by element at every
    angle by test_poles_and_near_poles."""
    import torch
    w = _near_pole_workload(frame, bf16, 61 + 2 * bf16 + (frame == "cos"))
    L, n = w.n_lobes, w.n
    P = w.params.shape[0]
    dt = torch.bfloat16 if bf16 else torch.float32
    params, c0 = _dev(w.params).to(dt), _dev(w.c0).to(dt)
    means, g_rgb = _dev(w.means), _dev(w.g_rgb)

    def bwd(p_, c_, m_, cm_):
        gp_, _, gm_ = ong.backward(p_, c_, m_, cm_, w.g_rgb, L, frame)
        return np.concatenate([gp_.ravel(), gm_.ravel()])

    ref, nu = sensitivity_floor(bwd, (w.params, w.c0, w.means, w.cam), (0, 1, 2, 3), draws=8, ulps=8)
    groups = np.concatenate([np.repeat(np.arange(P), n * L), np.full(3 * n, P)])
    prim = np.concatenate([np.tile(np.repeat(np.arange(n), L), P), np.repeat(np.arange(n), 3)])
    angle = np.repeat(NEAR_POLE_ANGLES, n // len(NEAR_POLE_ANGLES))
    resolved = np.isin(angle[prim], [1e-3, 1e-5])
    scale = np.array([np.abs(ref[groups == g]).max() for g in range(P + 1)])
    floor = _chain_floor(w.params, w.means, w.cam, w.g_rgb, L, frame)
    assert np.isfinite(floor[resolved]).all()
    atol = 1e-12 * scale[groups] + floor
    big = torch.empty(params.numel() + 16, device="cuda", dtype=dt)
    shifted = big[2:2 + params.numel()].view(params.shape)   # off the staged kernel's alignment
    shifted.copy_(params)
    runs = {
        "fused": lib.nasgabor_fused_fwd_bwd(params, c0, means, w.cam, g_rgb, L, frame_mode=frame),
        "bwd": (None,) + lib.nasgabor_eval_bwd(params, means, w.cam, g_rgb, L, frame_mode=frame),
        "register_path": (None,) + lib.nasgabor_eval_bwd(shifted, means, w.cam, g_rgb, L, frame_mode=frame),
    }
    lib.nasg_device_status()
    for name, out in runs.items():
        got = np.concatenate([out[1].cpu().numpy().ravel(), out[3].cpu().numpy().ravel()])
        assert np.isfinite(got).all(), name
        rep = grad_report(got[resolved], ref[resolved], nu[resolved], atol=atol[resolved])
        assert rep["violations"] == 0, (name, rep)
    # colours at the same directions
    _check_forward(lib, w, bf16)


def test_large_workload_sampled(lib):
    """N = 1e6, L = 8 (the single-scene throughput workload), FP32 and BF16, in the
    launch configuration the benchmark times; the oracle checks a seeded sample."""
    import torch
    n, L = 1_000_000, 8
    w = inputs.point_cloud_workload(n, L, 1002)
    sample = inputs.subsample_indices(n, 20_000, 1)
    for bf16 in (False, True):
        params, c0, p_np, c0_np = _prepare(w, bf16)
        means, g_rgb = _dev(w.means), _dev(w.g_rgb)
        rgb, g_p, g_c0, g_mu = lib.nasgabor_fused_fwd_bwd(params, c0, means, w.cam, g_rgb, L)
        torch.cuda.synchronize()
        lobes = (sample[:, None] * L + np.arange(L)).reshape(-1)
        ps, cs = p_np[:, lobes], c0_np[:, sample]
        ms, gs = w.means[sample], w.g_rgb[sample]

        def fwd(p, c, m, cam):
            return ong.forward(p, c, m, cam, L)

        ref, nu = sensitivity_floor(fwd, (ps, cs, ms, w.cam), (0, 1, 2, 3))
        rep = colour_report(rgb.cpu().numpy()[sample], ref, nu, COLOUR_BASE)
        assert rep["violations"] == 0, rep
        r_p, _, r_mu = ong.backward(ps, cs, ms, w.cam, gs, L)
        gp = g_p.cpu().numpy()[:, lobes]
        errs = [rel_l2(gp[p], r_p[p]) for p in range(10)]
        assert max(errs) <= GRAD_TOL, errs
        assert rel_l2(g_mu.cpu().numpy()[sample], r_mu) <= GRAD_TOL
        for t in (rgb, g_p, g_c0, g_mu):
            assert torch.isfinite(t).all()


def test_autograd_function(lib):
    import torch
    w = inputs.point_cloud_workload(1500, 4, 23)
    params = _dev(w.params).requires_grad_(True)
    c0 = _dev(w.c0).requires_grad_(True)
    means = _dev(w.means).requires_grad_(True)
    g = _dev(w.g_rgb)
    rgb = lib.NasgEval.apply(params, c0, means, tuple(w.cam.tolist()), 4)
    rgb.backward(g)
    gp, gc, gm = lib.nasgabor_eval_bwd(params.detach(), means.detach(), w.cam, g, 4)
    torch.testing.assert_close(params.grad, gp, rtol=0, atol=0)
    torch.testing.assert_close(c0.grad, gc, rtol=0, atol=0)
    torch.testing.assert_close(means.grad, gm, rtol=0, atol=0)


def test_empty_problem(lib):
    import torch
    z = torch.zeros((10, 0), device="cuda")
    out = lib.nasgabor_eval_fwd(z, torch.zeros((3, 0), device="cuda"), torch.zeros((0, 3), device="cuda"),
                                (0, 0, 3), 4)
    assert out.shape == (0, 3)
    g = lib.nasgabor_eval_bwd(z, torch.zeros((0, 3), device="cuda"), (0, 0, 3), torch.zeros((0, 3), device="cuda"), 4)
    assert g[0].shape == (10, 0)
    assert lib.sh_eval_fwd(torch.zeros((16, 3, 0), device="cuda"), torch.zeros((0, 3), device="cuda"),
                           (0, 0, 3)).shape == (0, 3)


def test_bounded_wait_reports_device_error(lib):
    """A kernel whose barrier never completes gives up after its iteration limit and
    sets the device error word; the context stays usable."""
    import torch
    lib.nasg_device_status()  # clear
    lib.nasg_probe_wait_timeout(1024)
    with pytest.raises(lib.NasgError) as ei:
        lib.nasg_device_status()
    assert ei.value.status == -6
    lib.nasg_device_status()  # cleared by the previous query
    x = torch.ones(16, device="cuda")
    assert float((x * 2).sum()) == 32.0


def test_bounded_wait_time(lib):
    """The longest wait the probe allows (2^20 tries) ends on its own, in at most the
    one-second wall-time bound plus the rounds before the next timer check; the time per
    try (the hardware's suspension interval) gives the worst case of the kernels' 2^22."""
    import torch
    lib.nasg_device_status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lib.nasg_probe_wait_timeout(1 << 20)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    with pytest.raises(lib.NasgError):
        lib.nasg_device_status()
    print(f"bounded wait: 2^20 tries in {ms:.3f} ms, {ms * 1e6 / 2 ** 20:.1f} ns per try")
    assert ms < 1500.0


@pytest.mark.parametrize("bf16,n,L", [(True, 4096, 8), (False, 4096, 8), (True, 1000, 4), (True, 2056, 16),
                                      (False, 1048, 2), (True, 8, 8),
                                      # any N: diffuse-colour planes off 16-byte boundaries, buffer ends
                                      # inside a 16-byte unit (plain-load tails), single-tile cases
                                      (True, 1001, 8), (True, 1003, 16), (True, 1002, 4), (False, 1037, 4),
                                      (False, 65, 8), (True, 1, 8), (True, 7, 8), (False, 13, 2),
                                      (False, 10, 6), (True, 129, 32)])
def test_staged_path_matches_oracle(lib, bf16, n, L):
    """Sizes that take the bulk-copy staged kernel (even L, N L sizeof(T) a multiple
    of 16 bytes), with ragged last tiles, against the oracle; and the same against the
    register path (an offset view breaks the 16-byte alignment the staged kernel needs)."""
    import torch
    w = inputs.point_cloud_workload(n, L, 31 + n + L)
    _check_forward(lib, w, bf16)
    _check_backward(lib, w, bf16)
    params, c0, _, _ = _prepare(w, bf16)
    means, g_rgb = _dev(w.means), _dev(w.g_rgb)
    f = lib.nasgabor_fused_fwd_bwd(params, c0, means, w.cam, g_rgb, L)
    big = torch.empty(params.numel() + 16, device="cuda", dtype=params.dtype)
    shifted = big[2:2 + params.numel()].view(params.shape)   # 4 or 8 bytes off 16-byte alignment
    shifted.copy_(params)
    r = lib.nasgabor_fused_fwd_bwd(shifted, c0, means, w.cam, g_rgb, L)
    lib.nasg_device_status()
    torch.testing.assert_close(r[0], f[0], rtol=1e-6, atol=1e-6)
    fg, rg = f[1].cpu().numpy(), r[1].cpu().numpy()
    assert max(rel_l2(rg[p], fg[p]) for p in range(fg.shape[0])) < 1e-6


@pytest.mark.parametrize("bf16,n,L", [(True, 1001, 8), (False, 4096, 8), (True, 1003, 16)])
def test_staged_path_accumulate(lib, bf16, n, L):
    """The staged kernel (any N) with accumulate: a second backward adds its gradients to
    the first, bit for bit twice the single pass (same summation order); the fused pass's
    gradients equal the backward's (rgb from the forward)."""
    import torch
    w = inputs.point_cloud_workload(n, L, 70 + n + L)
    params, c0, _, _ = _prepare(w, bf16)
    means, g_rgb = _dev(w.means), _dev(w.g_rgb)
    g1 = lib.nasgabor_eval_bwd(params, means, w.cam, g_rgb, L)
    gp, gc, gm = torch.zeros_like(g1[0]), torch.zeros_like(g1[1]), torch.zeros_like(g1[2])
    for _ in range(2):
        lib.nasgabor_eval_bwd(params, means, w.cam, g_rgb, L, g_params=gp, g_c0=gc, g_means=gm, accumulate=True)
    rgb = lib.nasgabor_eval_fwd(params, c0, means, w.cam, L)
    f = lib.nasgabor_fused_fwd_bwd(params, c0, means, w.cam, g_rgb, L)
    lib.nasg_device_status()  # raises if a bounded wait gave up
    torch.testing.assert_close(gp, 2 * g1[0], rtol=0, atol=0)
    torch.testing.assert_close(gc, 2 * g1[1], rtol=0, atol=0)
    torch.testing.assert_close(gm, 2 * g1[2], rtol=0, atol=0)
    torch.testing.assert_close(f[0], rgb, rtol=1e-6, atol=1e-6)
    fg, bg = f[1].cpu().numpy(), g1[0].cpu().numpy()
    assert max(rel_l2(fg[p], bg[p]) for p in range(fg.shape[0])) < 1e-6


@pytest.mark.parametrize("pinned", ["all", "none", "some"])
@pytest.mark.parametrize("n,L,chunk,bf16", [(100_003, 8, 16384, True), (4096, 4, 1024, False), (777, 3, 64, True),
                                            (5000, 8, 8, False)])
def test_host_resident_fused_matches_device_fused(lib, n, L, chunk, bf16, pinned):
    """Host arrays give the device-resident fused pass's results: page-locked ones read
    and written in place by the kernel; when any array is pageable, all of them are
    streamed in chunks through the device (copies overlapping the kernel)."""
    import torch
    w = inputs.point_cloud_workload(n, L, 60 + L)
    params, c0, _, _ = _prepare(w, bf16)
    means, g_rgb = _dev(w.means), _dev(w.g_rgb)
    ref = lib.nasgabor_fused_fwd_bwd(params, c0, means, w.cam, g_rgb, L)
    count = iter(range(8))

    def pin(t):   # "some": every other array page-locked
        j = next(count)
        return t.pin_memory() if pinned == "all" or (pinned == "some" and j % 2 == 0) else t

    hp = [pin(params.cpu()), pin(c0.cpu()), pin(means.cpu()), pin(g_rgb.cpu())]
    out = tuple(pin(torch.empty(t.shape, dtype=torch.float32)) for t in ref)
    hf = lib.HostFused(n, L, params.dtype, chunk=chunk)
    hf(hp[0], hp[1], hp[2], w.cam, hp[3], out)
    torch.cuda.synchronize()
    torch.testing.assert_close(out[0], ref[0].cpu(), rtol=1e-6, atol=1e-6)
    gp, rp = out[1].numpy(), ref[1].cpu().numpy()
    assert max(rel_l2(gp[p], rp[p]) for p in range(gp.shape[0])) < 1e-6
    torch.testing.assert_close(out[2], ref[2].cpu(), rtol=0, atol=0)
    assert rel_l2(out[3].numpy(), ref[3].cpu().numpy()) < 1e-6


def test_offsets_past_2_to_31_sampled(lib):
    """N = 27e6, L = 8 BF16: P N L = 2.16e9 elements per parameter array, past 2^31, so
    the kernels take 64-bit offsets; the last 300 primitives and 300 random ones
    against the oracle (about 25 GB on the device)."""
    import torch
    n, L = 27_000_000, 8
    d = inputs.device_point_cloud(n, L, 77, "cuda")
    params = d["params"].to(torch.bfloat16)
    del d["params"]
    c0 = d["c0"].to(torch.bfloat16)
    means, g_rgb, cam = d["means"], d["g_rgb"], d["cam"]
    rgb, g_p, g_c0, g_mu = lib.nasgabor_fused_fwd_bwd(params, c0, means, cam, g_rgb, L)
    torch.cuda.synchronize()
    rng = np.random.default_rng(78)
    sample = np.unique(np.concatenate([np.arange(n - 300, n), rng.choice(n, 300, replace=False)]))
    s_t = torch.from_numpy(sample).cuda()
    lobes = (s_t[:, None] * L + torch.arange(L, device="cuda")).reshape(-1)
    ps = params[:, lobes].float().cpu().numpy()
    cs = c0[:, s_t].float().cpu().numpy()
    ms = means[s_t].cpu().numpy()
    gs = g_rgb[s_t].cpu().numpy()
    cam_np = np.asarray(cam, dtype=np.float32)

    def fwd(p, c, m, cm):
        return ong.forward(p, c, m, cm, L)

    ref, nu = sensitivity_floor(fwd, (ps, cs, ms, cam_np), (0, 1, 2, 3))
    rep = colour_report(rgb[s_t].cpu().numpy(), ref, nu, COLOUR_BASE)
    assert rep["violations"] == 0, rep
    r_p, _, r_mu = ong.backward(ps, cs, ms, cam_np, gs, L)
    gp = g_p[:, lobes].cpu().numpy()
    assert max(rel_l2(gp[p], r_p[p]) for p in range(10)) <= GRAD_TOL
    assert rel_l2(g_mu[s_t].cpu().numpy(), r_mu) <= GRAD_TOL
    np.testing.assert_array_equal(g_c0[:, s_t].cpu().numpy(), gs.T)
