"""Parity helpers shared by the GPU tests: the sensitivity floor of the FP64
oracle and the error statistics the tolerances are written against.

Colour tolerance (FP32): |c_gpu - c_oracle| <= base + 4 nu_i per output, where
nu_i is the oracle's own sensitivity floor: the largest change of the FP64
colour when every FP32 input (raw parameters, c0, means, camera) is moved by
one ulp in a random direction, over `draws` seeded draws. For BF16-stored
parameters the oracle is fed the dequantised values and the same FP32-ulp
floor is used with a 4e-3 base. Gradients: relative L2 error per parameter
plane (and for c0 and the means) <= 1e-4.
"""
import numpy as np


def ulp_perturb(x, rng):
    x = np.asarray(x, dtype=np.float32)
    up = np.nextafter(x, np.float32(np.inf))
    dn = np.nextafter(x, np.float32(-np.inf))
    return np.where(rng.random(x.shape) < 0.5, up, dn).astype(np.float32)


def sensitivity_floor(forward, args, perturb_idx, draws=4, seed=99):
    """max over draws of |forward(perturbed args) - forward(args)| (elementwise)."""
    rng = np.random.default_rng(seed)
    ref = forward(*args)
    nu = np.zeros_like(ref)
    for _ in range(draws):
        pa = list(args)
        for j in perturb_idx:
            pa[j] = ulp_perturb(args[j], rng)
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


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    if den == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / den)
