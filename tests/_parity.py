"""Parity helpers shared by the GPU tests: the sensitivity floor of the FP64
oracle and the error statistics the tolerances are written against.

Colour tolerance (FP32): |c_gpu - c_oracle| <= base + 4 nu_i per output, where
nu_i is the oracle's own sensitivity floor: the largest change of the FP64
colour when every FP32 input (raw parameters, c0, means, camera) is moved by
one ulp in a random direction, over `draws` seeded draws. For BF16-stored
parameters the oracle is fed the dequantised values, and the same FP32-ulp
floor and the same 1e-5 base are used (the arithmetic is FP32 in both cases;
the error of BF16 storage itself, against the FP32 master values, is a separate
quantity bounded in tests/test_gpu_accuracy_report.py). Gradients: relative L2
error per parameter plane (and for c0 and the means) <= 1e-4, and element by
element where a test asks for it (grad_report).
"""
import math

import numpy as np

from oracle import nasgabor as ong


def ulp_perturb(x, rng, ulps=1):
    """Every element moved by `ulps` FP32 ulps up or down (random direction)."""
    x = np.asarray(x, dtype=np.float32)
    up = rng.random(x.shape) < 0.5
    y = x.copy()
    for _ in range(ulps):
        y = np.where(up, np.nextafter(y, np.float32(np.inf)), np.nextafter(y, np.float32(-np.inf)))
    return y.astype(np.float32)


def sensitivity_floor(forward, args, perturb_idx, draws=4, seed=99, ulps=1):
    """max over draws of |forward(perturbed args) - forward(args)| (elementwise), every
    FP32 input moved by `ulps` ulps in a random direction."""
    rng = np.random.default_rng(seed)
    ref = forward(*args)
    nu = np.zeros_like(ref)
    for _ in range(draws):
        pa = list(args)
        for j in perturb_idx:
            pa[j] = ulp_perturb(args[j], rng, ulps)
        nu = np.maximum(nu, np.abs(forward(*pa) - ref))
    return ref, nu


def colour_report(gpu, ref, nu, base):
    err = np.abs(np.asarray(gpu, dtype=np.float64) - ref)
    bound = base + 4.0 * nu
    return {
        "max_abs": float(err.max()) if err.size else 0.0,
        "max_rel1": float((err / np.maximum(1.0, np.abs(ref))).max()) if err.size else 0.0,
        "frac_under_1e-5": float((err <= 1e-5).mean()) if err.size else 1.0,
        "violations": int((err > bound).sum()),
        "worst_excess": float((err - bound).max()) if err.size else 0.0,
    }


def grad_report(gpu, ref, nu, rtol=1e-4, atol=1e-20):
    """Element-wise gradient check: |g_gpu - g_ref| <= rtol |g_ref| + 4 nu + atol, with nu
    the oracle's sensitivity floor of each element (as for the colours); atol (scalar or
    per element) only absorbs values far below any gradient that matters."""
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    nu = np.asarray(nu, dtype=np.float64).ravel()
    err = np.abs(gpu - ref)
    bound = rtol * np.abs(ref) + 4.0 * nu + atol
    bad = np.flatnonzero(~(err <= bound))
    return {
        "violations": int(bad.size),
        "first": [(int(j), float(gpu[j]), float(ref[j]), float(nu[j])) for j in bad[:5]],
        "finite": bool(np.isfinite(gpu).all()),
        "max_rel": float((err / np.maximum(np.abs(ref), 1e-30)).max()) if err.size else 0.0,
        "frac_tight": float(np.mean(nu <= 1e-3 * np.abs(ref))) if err.size else 1.0,
    }


def adam_consistency(theta_gpu, theta_old, m_gpu, v_gpu, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                     rtol=1e-5):
    """The GPU's new parameter values against the bias-corrected Adam update (torch
    order) formed in FP64 from its own new moments m, v: per element
    |theta_gpu - theta_exp| <= ulp32(theta_exp) + rtol |theta_exp - theta_old|.
    Together with the moments checked against the oracle, this tests the update
    without the cancellation of (new - old): the FP32 rounding of the new value alone
    is up to ulp/2 ~ 2.4e-7 at |theta| ~ 7, i.e. 2.4e-4 of a 1e-3 step."""
    th = np.asarray(theta_gpu, dtype=np.float64).ravel()
    o = np.asarray(theta_old, dtype=np.float64).ravel()
    m = np.asarray(m_gpu, dtype=np.float64).ravel()
    v = np.asarray(v_gpu, dtype=np.float64).ravel()
    bc1 = 1.0 - beta1 ** t
    bc2 = 1.0 - beta2 ** t
    exp = o - (lr / bc1) * m / (np.sqrt(v) / math.sqrt(bc2) + eps)
    ulp = np.spacing(np.abs(exp).astype(np.float32)).astype(np.float64)
    err = np.abs(th - exp)
    bad = np.flatnonzero(~(err <= ulp + rtol * np.abs(exp - o)))
    return {"violations": int(bad.size), "first": [(int(j), float(th[j]), float(exp[j]), float(o[j])) for j in bad[:5]],
            "max_err_over_ulp": float((err / ulp).max()) if err.size else 0.0}


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    if den == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / den)


EPS32 = 2.0 ** -24


def chain_floor(params, means, cam, g_rgb, L, frame="quat", norm="approx", act_mode="raw", family="nasgabor",
                 roundings=8, frame_planes=True):
    """Per-element rounding floor of the gradients that are sums of terms of opposite sign:
    the frame planes (dLoss/dx, dLoss/dz through the frame Jacobian), the means
    (dLoss/dd through I - d d^T) and the carrier's k and phi planes. Each is a sum whose
    terms can be many orders larger than the result (near a pole dLoss/dd is almost radial: at 1e-5 rad from the
    anti-pole ~1e7 against a tangential part ~1), and FP32 forms every term to a few
    roundings of its own magnitude, so the error a correct FP32 evaluation makes is
    about `roundings` * 2^-24 * (sum of the terms' magnitudes), which the oracle's
    input sensitivity (a smooth function of the inputs) does not see. Returned in the
    layout of grad_report's inputs: the P parameter planes (N*L each; 0 outside the
    frame planes, and everywhere without `frame_planes`) then the means (3 N)."""
    n = means.shape[0]
    variant = family
    p64 = np.asarray(params, np.float64)
    act = ong.activate(ong.split_planes(p64, n, L, frame, variant), frame, act_mode, variant)
    x, z = ong._frames(act, frame)
    d, dist = ong.view_directions(means, cam)
    G, par = ong.lobe(d[:, None, :], x, z, act["lam"], act["a"], act["k"], norm, need_grad=True,
                      phi=act.get("phi"))
    g_G = np.abs(np.sum(np.asarray(g_rgb, np.float64)[:, None, :] * act["w"], axis=-1))   # (N, L)
    mx, mz = np.linalg.norm(par["x"], axis=-1), np.linalg.norm(par["z"], axis=-1)
    md = np.linalg.norm(par["d"], axis=-1)
    tol = roundings * EPS32
    F = (4 if frame == "quat" else 3) if frame_planes else 0
    floor = np.zeros(p64.shape)
    if frame == "quat" and frame_planes:
        # the kernel's dLoss/dq = (2/|q|^2)[gv d.(dx~/dq)/2 + gu d.(dz~/dq)/2 - q (gv v + gu u)]
        # (x~, z~ the quadratic forms of the axes): every term is at most (|gu| + |gv|) |q| in
        # size, and a component can be far smaller than them (the sum is tangent to q)
        gu = g_G * np.sum(par["z"] * d[:, None, :], axis=-1)
        gv = g_G * np.sum(par["x"] * d[:, None, :], axis=-1)
        qn = np.sqrt(np.sum(np.asarray(act["q"], np.float64) ** 2, axis=-1))
        term = (tol * 4.0 * (np.abs(gu) + np.abs(gv)) / qn).reshape(-1)
        for f in range(4):
            floor[f] = term
    for f in range(F):
        h = 1e-6 * np.maximum(1.0, np.abs(p64[f]))
        fr = []
        for sgn in (1.0, -1.0):
            pp = p64.copy()
            pp[f] += sgn * h
            fr.append(ong._frames(ong.activate(ong.split_planes(pp, n, L, frame, variant), frame, act_mode,
                                               variant), frame))
        hh = (2.0 * h).reshape(n, L)
        jx = np.linalg.norm(fr[0][0] - fr[1][0], axis=-1) / hh
        jz = np.linalg.norm(fr[0][1] - fr[1][1], axis=-1) / hh
        floor[f] = np.maximum(floor[f], (tol * g_G * (mx * jx + mz * jz)).reshape(-1))
    # the carrier's k and phi partials, dG/dk = G d ln C^-1/dk - C^-1 p E sin(k v + phi) v/2 and
    # dG/dphi = G d ln C^-1/dphi - C^-1 p E sin(k v + phi)/2: where k v is small the two terms
    # nearly cancel (the normalisation takes out what the carrier's shift puts in)
    fields = ong.variant_fields(variant)
    F0 = 4 if frame == "quat" else 3
    if "k" in fields:
        phi = act.get("phi")
        arg = act["k"] * np.sum(d[:, None, :] * x, axis=-1) + (0.0 if phi is None else phi)
        hh = (1.0 + np.cos(arg)) / 2.0
        cpe = np.where(hh > 0.0, G / np.where(hh > 0.0, hh, 1.0), 0.0)
        sn = np.sin(arg)
        vv = np.sum(d[:, None, :] * x, axis=-1)
        slopes = ong.activation_slopes(act, act_mode)
        t2 = -0.5 * cpe * sn * vv
        floor[F0 + fields.index("k")] = (tol * g_G * np.abs(slopes["k"]) * (np.abs(par["k"] - t2) + np.abs(t2))).reshape(-1)
        if "phi" in fields:
            t2 = -0.5 * cpe * sn
            floor[F0 + fields.index("phi")] = (tol * g_G * (np.abs(par["phi"] - t2) + np.abs(t2))).reshape(-1)
    # component c of (I - d d^T) g_d: the c-th terms of g_d and (g_d . d) d_c
    terms_c = np.sum(np.abs(g_G[..., None] * par["d"]), axis=1)                          # (N, 3)
    fm = tol * (terms_c + np.sum(g_G * md, axis=1)[:, None] * np.abs(d)) / dist[:, None]
    return np.concatenate([floor.ravel(), fm.ravel()])
