"""FP64 CPU oracle for the NASGabor appearance model.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import or call this
module: it exists so that tests, the smoke check and the CPU-baseline leg of the
benchmark can check the CUDA library against a plain, slow, obviously correct
restatement of the paper's definitions. It shares no code with the CUDA path.

Every quantity is computed in float64 from the float32 (or dequantised bfloat16)
inputs the GPU sees, step by step in the paper's notation, vectorised over
primitives and lobes with numpy (no blocking, fusion or reordering).

Sources (arXiv 2606.09794, "Beyond Spherical Harmonics"):
  * appearance model  f_C(d) = c0 + sum_l w_l G_l(d)            -- Sec. 4.2, eq:app_model
  * NASGabor kernel G, kappa, tau                               -- Sec. 5.1 (definition)
  * approximate normalisation C^-1 = lam sqrt(1+a) / (2 pi (1-e^{-2 lam}))
                                                                -- Supp. E/F, used by all
                                                                   Sec. 6 results (Sec. 5.1)
  * closed-form integral (1 + Psi) and Lambda = lam (1 + a)     -- Sec. 5.1 (integral)
  * activations (tanh, exp, exp, 20 (tanh + 1), tanh)           -- Supp. C, activation table
  * frame from cosines (z, x; y = z x x)                        -- Supp. C, parameterisation
  * derivatives wrt a, lam, x, z, k                             -- Supp. F
  * derivatives of the frame wrt the cosines                    -- Supp. E (auxiliary)
  * central-ray evaluation: one colour per primitive, at d = normalize(mu - cam)
                                                                -- Sec. 5.2 (impl. details)

Readings where the paper is silent, ambiguous or mistaken (each one is also
listed with its reason in the design notes):
  R1  normalised kernel: G = C^-1 p E h (Supp. F); norm_mode "none" drops C^-1
      (the Sec. 5.1 display). At d = z the normalised value is the limit C^-1.
  R2  poles: where 1 - u^2 == 0 (u = d.z), u > 0 takes tau := 0 (and zero
      derivatives of tau), giving G = C^-1 h(v); u < 0 gives G := 0 with all
      derivatives 0. 1 - u^2 is evaluated as |d x z|^2 (equal for unit d, z), and
      1 - u, 1 + u from it where each is small, so that the rule applies at the
      exact poles only and directions a little off them keep full accuracy
      (1 - u u in FP64 rounds to 0 within ~1.5e-8 rad of the axis and loses ~1 %
      at 1e-7 rad); likewise ln kappa by log1p near kappa = 1 and E kappa - 1 by
      expm1.
  R3  Supp. E writes ln(tau) in dp/da; the factor is ln(kappa) (as in Supp. F).
  R4  dC^-1/dlam printed with "+ 2 lam sqrt(1+a) e^{-2 lam}" in the numerator;
      differentiating C^-1 gives "-". The minus sign is used (pinned by finite
      differences in the tests).
  R5  the epsilon in (1 + eps - e^{-2 lam}) is undefined: eps = 0.
  R6  the derivatives are taken wrt the activated quantities and chained through
      the Supp. C activations to the stored raw values.
  R7  Supp. E names the in-plane angle psi; Supp. C calls it tau. Same parameter.
  R8  the paper gives no dG/dd. G depends on d only through u = d.z and v = d.x,
      so dG/dd = (dG/dv) x + (dG/du) z, with dG/dx = (dG/dv) d and
      dG/dz = (dG/du) d read off the Supp. F vector formulas.
  R9  QUAT frame mode (not in the paper): x and z are the first and third
      columns of the rotation matrix of the normalised quaternion (w, x, y, z).
  R10 variants: NASG is the lobe with k = 0 (no carrier), SG the lobe with a = 0
      and k = 0 (the isotropic normalised spherical Gaussian of the distributions
      table), "phase" the lobe with the carrier (1 + cos(k v + phi))/2 and a
      per-lobe phase phi stored without activation. Its integral: the envelope
      is even in v, so the sin(k v) sin(phi) part integrates to zero and the
      closed form becomes pi (1 - e^{-2 lam}) / (lam sqrt(1+a)) (1 + cos(phi) Psi).
"""
from __future__ import annotations

import math

import numpy as np

FRAME_QUAT = "quat"
FRAME_COS = "cos"
NORM_APPROX = "approx"
NORM_NONE = "none"
NORM_EXACT = "exact"
ACT_RAW = "raw"
ACT_IDENTITY = "identity"


VAR_NASGABOR = "nasgabor"
VAR_NASG = "nasg"
VAR_SG = "sg"
VAR_PHASE = "phase"

# per-lobe scalars after the frame, in storage order (R10)
_FIELDS = {
    VAR_NASGABOR: ("lam", "a", "k", "w0", "w1", "w2"),
    VAR_NASG: ("lam", "a", "w0", "w1", "w2"),
    VAR_SG: ("lam", "w0", "w1", "w2"),
    VAR_PHASE: ("lam", "a", "k", "phi", "w0", "w1", "w2"),
}


def variant_fields(variant: str = VAR_NASGABOR):
    return _FIELDS[variant]


def lobe_planes(frame_mode: str, variant: str = VAR_NASGABOR) -> int:
    return (4 if frame_mode == FRAME_QUAT else 3) + len(_FIELDS[variant])


# ---------------------------------------------------------------------------
# View direction (Sec. 5.2: one evaluation per primitive along the central ray)
# ---------------------------------------------------------------------------

def view_directions(means, cam):
    """d_i = (mu_i - cam) / |mu_i - cam| in float64; also returns |mu_i - cam|."""
    r = np.asarray(means, dtype=np.float64) - np.asarray(cam, dtype=np.float64)[None, :]
    dist = np.sqrt(np.sum(r * r, axis=-1))
    return r / dist[:, None], dist


# ---------------------------------------------------------------------------
# Activations (Supp. C, activation table)
# ---------------------------------------------------------------------------

def split_planes(params, n, n_lobes, frame_mode, variant=VAR_NASGABOR):
    """params [P][N*L] -> float64 array (P, N, L)."""
    p = np.asarray(params, dtype=np.float64)
    return p.reshape(lobe_planes(frame_mode, variant), n, n_lobes)


def activate(planes, frame_mode, act_mode=ACT_RAW, variant=VAR_NASGABOR):
    """Map raw planes (P, N, L) to the activated lobe quantities.

    Returns a dict with lam, a, k, phi (N, L), w (N, L, 3), and the frame inputs:
    QUAT: q (N, L, 4); COS: c (N, L, 3) cosines of theta, phi, tau. Quantities a
    variant does not store are 0 (R10); the carrier phase is stored as is.
    """
    out = {}
    if frame_mode == FRAME_QUAT:
        out["q"] = np.moveaxis(planes[0:4], 0, -1)
        rest = planes[4:]
    else:
        frame_raw = np.moveaxis(planes[0:3], 0, -1)
        out["c_raw"] = frame_raw
        out["c"] = frame_raw if act_mode == ACT_IDENTITY else np.tanh(frame_raw)
        # the sines s = sqrt(1 - c^2) >= 0; for c = tanh r that is sech r = 1/cosh r, which
        # keeps its relative accuracy where tanh r is within rounding of +-1
        out["s"] = np.sqrt(1.0 - out["c"] ** 2) if act_mode == ACT_IDENTITY else 1.0 / np.cosh(frame_raw)
        rest = planes[3:]
    f = {name: rest[j] for j, name in enumerate(_FIELDS[variant])}
    lam_r = f["lam"]
    zero = np.zeros_like(lam_r)
    w_r = np.stack([f["w0"], f["w1"], f["w2"]], axis=-1)
    if act_mode == ACT_IDENTITY:
        out["lam"], out["w"] = lam_r, w_r
        out["a"] = f.get("a", zero)
        out["k"] = f.get("k", zero)
    else:
        out["lam"] = np.exp(lam_r)
        out["a"] = np.exp(f["a"]) if "a" in f else zero
        out["k"] = 20.0 * (np.tanh(f["k"]) + 1.0) if "k" in f else zero
        out["w"] = np.tanh(w_r)
    out["phi"] = f.get("phi", zero)
    out["raw"] = {"lam": lam_r, "a": f.get("a", zero), "k": f.get("k", zero), "w": w_r}
    return out


def activation_slopes(act, act_mode):
    """d(activated)/d(raw) for lam, a, k, w (Supp. C activations differentiated)."""
    one = np.ones_like(act["lam"])
    if act_mode == ACT_IDENTITY:
        return {"lam": one, "a": one, "k": one, "phi": one, "w": np.ones_like(act["w"])}
    t = np.tanh(act["raw"]["k"])
    return {
        "lam": act["lam"],                 # d exp(r)/dr
        "a": act["a"],                     # d exp(r)/dr
        "k": 20.0 * (1.0 - t * t),         # d 20 (tanh r + 1)/dr
        "phi": one,                        # stored as is
        "w": 1.0 - act["w"] ** 2,          # d tanh r/dr
    }


# ---------------------------------------------------------------------------
# Frames
# ---------------------------------------------------------------------------

def frame_from_quat(q):
    """R9: x = R(q^) e_x, z = R(q^) e_z for the unit quaternion q^ = q/|q| = (w, x, y, z)."""
    qn = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = (qn[..., j] for j in range(4))
    xa = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], axis=-1)
    za = np.stack([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], axis=-1)
    return xa, za


def _quat_frame_jacobians(q):
    """d x / d q and d z / d q (shape (..., 3, 4)) including the normalisation q -> q/|q|."""
    nq = np.linalg.norm(q, axis=-1, keepdims=True)
    qn = q / nq
    w, x, y, z = (qn[..., j] for j in range(4))
    zero = np.zeros_like(w)
    # Partials of the unit-quaternion formulas wrt (w, x, y, z), columns in that order.
    dx = np.stack([
        np.stack([zero, zero, -4 * y, -4 * z], axis=-1),
        np.stack([2 * z, 2 * y, 2 * x, 2 * w], axis=-1),
        np.stack([-2 * y, 2 * z, -2 * w, 2 * x], axis=-1),
    ], axis=-2)
    dz = np.stack([
        np.stack([2 * y, 2 * z, 2 * w, 2 * x], axis=-1),
        np.stack([-2 * x, -2 * w, 2 * z, 2 * y], axis=-1),
        np.stack([zero, -4 * x, -4 * y, zero], axis=-1),
    ], axis=-2)
    # d q^/d q = (I - q^ q^T)/|q|
    eye = np.eye(4)
    proj = (eye - qn[..., :, None] * qn[..., None, :]) / nq[..., None]
    return dx @ proj, dz @ proj


def frame_from_cos(c, s=None):
    """Supp. C: z = (ct sp, st sp, cp), x = (ct cp cs - st ss, st cp cs + ct ss, -sp cs);
    s = sqrt(1 - c^2) unless the sines are given."""
    ct, cp, cs = c[..., 0], c[..., 1], c[..., 2]
    if s is None:
        s = np.sqrt(1.0 - c * c)
    st, sp, ss = s[..., 0], s[..., 1], s[..., 2]
    za = np.stack([ct * sp, st * sp, cp], axis=-1)
    xa = np.stack([ct * cp * cs - st * ss, st * cp * cs + ct * ss, -sp * cs], axis=-1)
    return xa, za


def _cos_frame_partials(c, s=None):
    """Partials of x and z wrt the six quantities (ct, st, cp, sp, cs, ss), each a 3-vector.

    The Supp. E formulas for dx/dc, dz/dc are these partials combined with
    ds/dc = -c/s; they are combined here with the chosen chain (raw or identity).
    """
    ct, cp, cs = c[..., 0], c[..., 1], c[..., 2]
    if s is None:
        s = np.sqrt(1.0 - c * c)
    st, sp, ss = s[..., 0], s[..., 1], s[..., 2]
    zero = np.zeros_like(ct)
    vx = lambda a, b, d: np.stack([a, b, d], axis=-1)  # noqa: E731
    px = {
        "ct": vx(cp * cs, ss, zero), "st": vx(-ss, cp * cs, zero),
        "cp": vx(ct * cs, st * cs, zero), "sp": vx(zero, zero, -cs),
        "cs": vx(ct * cp, st * cp, -sp), "ss": vx(-st, ct, zero),
    }
    pz = {
        "ct": vx(sp, zero, zero), "st": vx(zero, sp, zero),
        "cp": vx(zero, zero, np.ones_like(ct)), "sp": vx(ct, st, zero),
        "cs": vx(zero, zero, zero), "ss": vx(zero, zero, zero),
    }
    return px, pz, (ct, st, cp, sp, cs, ss)


# ---------------------------------------------------------------------------
# The lobe (Sec. 5.1 definition; Supp. F factorisation G = C^-1 p E h)
# ---------------------------------------------------------------------------

def norm_approx(lam, a):
    """Supp. E/F: C^-1 = lam sqrt(1+a) / (2 pi (1 - e^{-2 lam}))."""
    return lam * np.sqrt(1.0 + a) / (2.0 * np.pi * (1.0 - np.exp(-2.0 * lam)))


def _exp_sinhc(big, k):
    """e^{-Lambda} sinhc(sqrt(Lambda^2 - k^2)) for real or complex arguments.

    sinhc(s) = sinh(s)/s is an entire function of sigma = s^2 = Lambda^2 - k^2:
    for sigma > 0 the product is (e^{s - Lambda} - e^{-s - Lambda}) / (2 s) with
    s - Lambda = -k^2 / (s + Lambda) (the same value; no overflow of sinh at
    Lambda up to 2e3); for sigma < 0, with t = sqrt(-sigma), it is
    e^{-Lambda} sin(t)/t; near sigma = 0 its Taylor series in sigma. Each branch is
    analytic, so the complex-step derivatives below go through it."""
    big = np.asarray(big)
    k = np.asarray(k)
    sigma = (big - k) * (big + k)
    small = np.abs(sigma) < 1e-3
    pos = np.real(sigma) > 0
    one = np.ones_like(sigma)
    sig_p = np.where(pos & ~small, sigma, one)
    s = np.sqrt(sig_p)
    br_pos = (np.exp(-(k * k) / (s + big)) - np.exp(-s - big)) / (2.0 * s)
    sig_n = np.where(~pos & ~small, -sigma, one)
    t = np.sqrt(sig_n)
    br_neg = np.exp(-big) * np.sin(t) / t
    br_small = np.exp(-big) * (1.0 + sigma * (1.0 / 6.0 + sigma * (1.0 / 120.0 + sigma * (
        1.0 / 5040.0 + sigma / 362880.0))))
    return np.where(small, br_small, np.where(pos, br_pos, br_neg))


def integral_closed_form(lam, a, k, phi=0.0):
    """Sec. 5.1: int G = pi (1 - e^{-2 lam}) / (lam sqrt(1+a)) (1 + Psi),
    Psi = 2 Lambda e^{-Lambda} sinhc(sqrt(Lambda^2 - k^2)) / (1 - e^{-2 Lambda}), Lambda = lam (1+a),
    sinhc(s) = sinh(s)/s, continued to sin(|s|)/|s| for imaginary s (k > Lambda) and 1 at s = 0.
    The product e^{-Lambda} sinhc is formed without overflow (_exp_sinhc). With a
    carrier phase phi (R10) Psi is multiplied by cos(phi)."""
    lam = np.asarray(lam, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    big = lam * (1.0 + a)
    psi = 2.0 * big * _exp_sinhc(big, k) / (1.0 - np.exp(-2.0 * big))
    return np.pi * (1.0 - np.exp(-2.0 * lam)) / (lam * np.sqrt(1.0 + a)) * (1.0 + np.cos(phi) * psi)


def lobe(d, x, z, lam, a, k, norm_mode=NORM_APPROX, need_grad=False, phi=None):
    """G(d; [x, y, z], lam, a, k) and, optionally, its Supp. F partials.

    Shapes: d, x, z (..., 3); lam, a, k (...); phi (...) the carrier phase (R10,
    default 0). Returns G, or (G, partials) with partials = dict(x=dG/dx,
    z=dG/dz, d=dG/dd (vectors), lam, a, k, phi (scalars)).
    """
    if phi is None:
        phi = np.zeros_like(np.asarray(lam, dtype=np.float64))
    u = np.sum(d * z, axis=-1)
    v = np.sum(d * x, axis=-1)
    # 1 - u^2 = |d x z|^2 for unit d, z (the same number, without the cancellation of
    # 1 - u u near the poles); 1 - u and 1 + u from it on the side where each is small
    dz = np.cross(d, z)
    one_m_u2 = np.sum(dz * dz, axis=-1)
    pole = one_m_u2 <= 0.0
    safe = np.where(pole, 1.0, one_m_u2)
    up = u >= 0.0
    one_m_u = np.where(up, safe / np.where(up, 1.0 + u, 1.0), 1.0 - u)
    one_p_u = np.where(up, 1.0 + u, safe / np.where(up, 1.0, 1.0 - u))
    kappa = one_p_u / 2.0
    kappa_safe = np.where(pole, 1.0, kappa)
    tau = np.where(pole, 0.0, a * v * v / safe)
    # ln kappa = log1p(-(1 - u)/2) where kappa is near 1; E kappa - 1 = expm1((1 + tau) ln kappa)
    ln_kappa = np.where(pole, 0.0, np.where(up, np.log1p(-np.minimum(one_m_u, 1.0) / 2.0),
                                            np.log(np.where(kappa_safe > 0.0, kappa_safe, 1.0))))
    E = np.exp(tau * ln_kappa)
    ek_m1 = np.expm1((1.0 + tau) * ln_kappa)
    p = np.exp(2.0 * lam * ek_m1)
    h = (1.0 + np.cos(k * v + phi)) / 2.0
    if norm_mode == NORM_NONE:
        cinv = np.ones_like(lam)
    elif norm_mode == NORM_APPROX:
        cinv = norm_approx(lam, a)
    elif norm_mode == NORM_EXACT:
        cinv = 1.0 / integral_closed_form(lam, a, k, phi)
    else:
        raise ValueError(norm_mode)
    anti = pole & (u < 0.0)
    G = np.where(anti, 0.0, p * E * cinv * h)
    if not need_grad:
        return G

    # --- Supp. F partial derivatives (readings R3-R5, R8) ---
    dvec = d
    # wrt a
    dtau_da = np.where(pole, 0.0, v * v / safe)
    dp_da = p * (2.0 * lam * E * kappa_safe) * ln_kappa * dtau_da
    dE_da = E * ln_kappa * dtau_da
    if norm_mode == NORM_APPROX:
        dcinv_da = lam / (2.0 * np.sqrt(1.0 + a)) / (2.0 * np.pi * (1.0 - np.exp(-2.0 * lam)))
        em = np.exp(-2.0 * lam)
        dcinv_dlam = (np.sqrt(1.0 + a) * (1.0 - em) - 2.0 * lam * np.sqrt(1.0 + a) * em) / (
            2.0 * np.pi * (1.0 - em) ** 2)
        dcinv_dk = np.zeros_like(lam)
        dcinv_dphi = np.zeros_like(lam)
    elif norm_mode == NORM_NONE:
        dcinv_da = np.zeros_like(lam)
        dcinv_dlam = np.zeros_like(lam)
        dcinv_dk = np.zeros_like(lam)
        dcinv_dphi = np.zeros_like(lam)
    else:
        dcinv_dlam, dcinv_da, dcinv_dk, dcinv_dphi = _exact_norm_partials(lam, a, k, phi)
    dG_da = (dp_da * E * cinv + p * dE_da * cinv + p * E * dcinv_da) * h
    # wrt lam
    dp_dlam = 2.0 * p * ek_m1
    dG_dlam = (E * cinv * dp_dlam + E * p * dcinv_dlam) * h
    # wrt x: dtau/dx = 2 a v/(1-u^2) d ; dE/dx = E ln(kappa) dtau/dx ; dp/dx = 2 lam p kappa dE/dx
    coef_tau_x = np.where(pole, 0.0, 2.0 * a * v / safe)
    coef_E_x = E * ln_kappa * coef_tau_x
    coef_p_x = 2.0 * lam * p * kappa_safe * coef_E_x
    coef_h_x = -(k / 2.0) * np.sin(k * v + phi)
    dG_dv = (coef_p_x * E * cinv + p * coef_E_x * cinv) * h + p * E * cinv * coef_h_x
    # wrt z: dkappa/dz = d/2 ; dtau/dz = a v^2 2u/(1-u^2)^2 d
    coef_kappa_z = 0.5
    coef_tau_z = np.where(pole, 0.0, a * v * v * 2.0 * u / (safe * safe))
    coef_E_z = E * (tau / kappa_safe * coef_kappa_z + ln_kappa * coef_tau_z)
    coef_p_z = p * 2.0 * lam * (kappa_safe * coef_E_z + E * coef_kappa_z)
    dG_du = (coef_p_z * E * cinv + p * coef_E_z * cinv) * h
    # wrt k
    dG_dk = p * E * cinv * (-(v / 2.0) * np.sin(k * v + phi)) + p * E * h * dcinv_dk
    # wrt the carrier phase (R10)
    dG_dphi = p * E * cinv * (-0.5 * np.sin(k * v + phi)) + p * E * h * dcinv_dphi
    zero = lambda t: np.where(anti, 0.0, t)  # noqa: E731
    dG_du, dG_dv = zero(dG_du), zero(dG_dv)
    partials = {
        "x": dG_dv[..., None] * dvec,
        "z": dG_du[..., None] * dvec,
        "d": dG_dv[..., None] * x + dG_du[..., None] * z,
        "lam": zero(dG_dlam),
        "a": zero(dG_da),
        "k": zero(dG_dk),
        "phi": zero(dG_dphi),
    }
    return G, partials


def _exact_norm_partials(lam, a, k, phi=0.0):
    """Partials of 1/int G (Sec. 5.1 closed form) wrt lam, a, k, phi by the complex-step method.

    The complex step evaluates the closed form at (value + i h) and reads the
    derivative from the imaginary part; it has no subtractive cancellation, so
    it is accurate to working precision for the analytic closed form.
    """
    h = 1e-30
    out = []
    for which in range(4):
        args = [np.asarray(lam, dtype=np.complex128), np.asarray(a, dtype=np.complex128),
                np.asarray(k, dtype=np.complex128), np.asarray(phi, dtype=np.complex128)]
        args[which] = args[which] + 1j * h
        val = _integral_closed_form_complex(*args)
        out.append(np.imag(1.0 / val) / h)
    return out[0], out[1], out[2], out[3]


def _integral_closed_form_complex(lam, a, k, phi):
    big = lam * (1.0 + a)
    psi = 2.0 * big * _exp_sinhc(big, k) / (1.0 - np.exp(-2.0 * big))
    return np.pi * (1.0 - np.exp(-2.0 * lam)) / (lam * np.sqrt(1.0 + a)) * (1.0 + np.cos(phi) * psi)


# ---------------------------------------------------------------------------
# Whole model: forward and backward over N primitives with L lobes each
# ---------------------------------------------------------------------------

def _frames(act, frame_mode):
    if frame_mode == FRAME_QUAT:
        return frame_from_quat(act["q"])
    return frame_from_cos(act["c"], act.get("s"))


def forward(params, c0, means, cam, n_lobes, frame_mode=FRAME_QUAT, norm_mode=NORM_APPROX,
            act_mode=ACT_RAW, variant=VAR_NASGABOR):
    """f_C(d_i) = c0_i + sum_l w_il G_il(d_i) for every primitive (eq:app_model); (N, 3) float64."""
    means = np.asarray(means)
    n = means.shape[0]
    planes = split_planes(params, n, n_lobes, frame_mode, variant)
    act = activate(planes, frame_mode, act_mode, variant)
    d, _ = view_directions(means, cam)
    x, z = _frames(act, frame_mode)
    G = lobe(d[:, None, :], x, z, act["lam"], act["a"], act["k"], norm_mode, phi=act["phi"])
    c0 = np.asarray(c0, dtype=np.float64)
    return c0.T + np.sum(act["w"] * G[..., None], axis=1)


def backward(params, c0, means, cam, g_rgb, n_lobes, frame_mode=FRAME_QUAT,
             norm_mode=NORM_APPROX, act_mode=ACT_RAW, variant=VAR_NASGABOR):
    """Gradients of <g_rgb, f_C> wrt the raw lobe planes, c0 and the means.

    Returns (g_params (P, N*L), g_c0 (3, N), g_means (N, 3)), float64.
    """
    means = np.asarray(means)
    n = means.shape[0]
    g_rgb = np.asarray(g_rgb, dtype=np.float64)
    planes = split_planes(params, n, n_lobes, frame_mode, variant)
    act = activate(planes, frame_mode, act_mode, variant)
    slope = activation_slopes(act, act_mode)
    d, dist = view_directions(means, cam)
    x, z = _frames(act, frame_mode)
    G, par = lobe(d[:, None, :], x, z, act["lam"], act["a"], act["k"], norm_mode, need_grad=True, phi=act["phi"])

    g_c = g_rgb[:, None, :]                                    # (N, 1, 3)
    g_w = g_c * G[..., None]                                   # dL/dw_l
    g_G = np.sum(g_c * act["w"], axis=-1)                      # dL/dG_l
    grads = {
        "lam": g_G * par["lam"] * slope["lam"],
        "a": g_G * par["a"] * slope["a"],
        "k": g_G * par["k"] * slope["k"],
        "phi": g_G * par["phi"] * slope["phi"],
        "w": g_w * slope["w"],
    }
    g_x = g_G[..., None] * par["x"]
    g_z = g_G[..., None] * par["z"]
    if frame_mode == FRAME_QUAT:
        jx, jz = _quat_frame_jacobians(act["q"])
        g_q = np.einsum("nli,nlij->nlj", g_x, jx) + np.einsum("nli,nlij->nlj", g_z, jz)
        frame_planes = [g_q[..., j] for j in range(4)]
    else:
        px, pz, (ct, st, cp, sp, cs, ss) = _cos_frame_partials(act["c"], act.get("s"))
        if act_mode == ACT_IDENTITY:
            # d/dc with ds/dc = -c/s (Supp. E)
            dc = {"t": (1.0, -ct / st), "p": (1.0, -cp / sp), "s": (1.0, -cs / ss)}
        else:
            # raw r with c = tanh r: dc/dr = 1 - c^2 = s^2 and s = sech r, ds/dr = -c s
            dc = {"t": (st * st, -ct * st), "p": (sp * sp, -cp * sp), "s": (ss * ss, -cs * ss)}
        frame_planes = []
        for ang, (cn, sn) in (("t", ("ct", "st")), ("p", ("cp", "sp")), ("s", ("cs", "ss"))):
            dcdr, dsdr = dc[ang]
            dxr = px[cn] * np.asarray(dcdr)[..., None] + px[sn] * np.asarray(dsdr)[..., None]
            dzr = pz[cn] * np.asarray(dcdr)[..., None] + pz[sn] * np.asarray(dsdr)[..., None]
            frame_planes.append(np.sum(g_x * dxr, axis=-1) + np.sum(g_z * dzr, axis=-1))
    per_field = {"lam": grads["lam"], "a": grads["a"], "k": grads["k"], "phi": grads["phi"],
                 "w0": grads["w"][..., 0], "w1": grads["w"][..., 1], "w2": grads["w"][..., 2]}
    out_planes = frame_planes + [per_field[name] for name in _FIELDS[variant]]
    g_params = np.stack([pl.reshape(-1) for pl in out_planes])
    g_c0 = g_rgb.T.copy()
    g_d = np.sum(g_G[..., None] * par["d"], axis=1)            # (N, 3)
    # d = r/|r|: dL/dmu = (I - d d^T) dL/dd / |r|
    g_means = (g_d - np.sum(g_d * d, axis=-1, keepdims=True) * d) / dist[:, None]
    return g_params, g_c0, g_means
