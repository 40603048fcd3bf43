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
