"""Seeded synthetic workloads for the NASGabor appearance path.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's
tests. It holds no arithmetic of the method itself: it only draws random
numbers and lays them out in the buffers the library consumes.

Parameters are drawn in the *activated* space the workloads are specified in
(sharpness lambda log-uniform in [1, 1e3], anisotropy a ~ U[0, 1], Gabor
frequency k ~ U[0, 8], RGB amplitude w ~ U[0, 1]^3, frame quaternion uniform on
S^3) and stored as the *raw* values the model activates (Supp. C table:
lambda = exp(r), a = exp(r), k = 20 (tanh r + 1), w = tanh r), i.e. by
inverse-transform sampling of the raw variables.

Every workload is a pure function of its seed. Substreams are spawned from one
``numpy.random.SeedSequence`` in a fixed order (positions, quat, lambda, a, k,
phase, w, c0, upstream gradient / SH coefficients), so adding a draw to one
substream never shifts another.

Layouts (shared with include/nasgabor.h):
  params  [P][N*L] float32, plane-major, lobe-minor (index p*N*L + i*L + l)
          QUAT planes: q_w q_x q_y q_z lam_r a_r k_r w_r w_g w_b   (P = 10)
          COS  planes: ct_r cp_r cpsi_r lam_r a_r k_r w_r w_g w_b  (P = 9)
  c0      [3][N] float32 (planar)
  means   [N][3] float32
  cam     [3]   float32
  g_rgb   [N][3] float32
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FRAME_QUAT = "quat"
FRAME_COS = "cos"

_SUBSTREAMS = ("positions", "quat", "lam", "a", "k", "phase", "w", "c0", "upstream")

# Clamps that keep the inverse-transformed raw values finite at the open ends
# of the activated ranges (a, k >= 1e-6; |w| <= 1 - 2^-20).
_A_MIN = 1e-6
_K_MIN = 1e-6
_W_MAX = 1.0 - 2.0 ** -20


def lobe_planes(frame_mode: str) -> int:
    """Raw scalars per lobe: 4 quaternion + 6 (QUAT) or 3 cosines + 6 (COS)."""
    if frame_mode == FRAME_QUAT:
        return 10
    if frame_mode == FRAME_COS:
        return 9
    raise ValueError(f"unknown frame mode {frame_mode!r}")


def _streams(seed: int) -> dict[str, np.random.Generator]:
    ss = np.random.SeedSequence(seed)
    kids = ss.spawn(len(_SUBSTREAMS))
    return {name: np.random.default_rng(kid) for name, kid in zip(_SUBSTREAMS, kids)}


@dataclasses.dataclass
class Workload:
    n: int
    n_lobes: int
    frame_mode: str
    params: np.ndarray        # (P, N*L) float32 raw parameters
    c0: np.ndarray            # (3, N) float32 diffuse colour
    means: np.ndarray         # (N, 3) float32 primitive centres
    cam: np.ndarray           # (3,) float32 camera centre
    g_rgb: np.ndarray | None  # (N, 3) float32 upstream gradient
    phase: np.ndarray | None  # (N*L,) float32 carrier phase draw (unused by the paper's G)

    @property
    def n_planes(self) -> int:
        return lobe_planes(self.frame_mode)


def _draw_lobes(st, count: int, frame_mode: str, k_max: float = 8.0, activated: bool = False):
    """Raw lobe parameters for `count` lobes, drawn by inverse transform.

    With activated=True the stored values are the activated quantities
    themselves (lam, a, k, w, and the frame cosines in COS mode)."""
    if frame_mode == FRAME_QUAT:
        q = st["quat"].standard_normal((count, 4))
        q /= np.linalg.norm(q, axis=1, keepdims=True)
        frame = [q[:, j] for j in range(4)]
    else:
        # Frame cosines: uniform angles theta in [0, pi), phi in [0, pi),
        # psi in [0, pi); the stored raw value is atanh(cos(angle)) so that
        # tanh(raw) reproduces the cosine. Angles are kept off the ends so
        # the raw values stay finite.
        ang = st["quat"].uniform(0.02, math.pi - 0.02, size=(count, 3))
        if activated:
            frame = [np.cos(ang[:, j]) for j in range(3)]
        else:
            frame = [np.arctanh(np.cos(ang[:, j])) for j in range(3)]
    lam = np.exp(st["lam"].uniform(0.0, math.log(1e3), size=count))
    lam_r = np.log(lam)
    a = np.maximum(st["a"].uniform(0.0, 1.0, size=count), _A_MIN)
    a_r = np.log(a)
    k = np.maximum(st["k"].uniform(0.0, k_max, size=count), _K_MIN)
    k_r = np.arctanh(k / 20.0 - 1.0)
    phase = st["phase"].uniform(0.0, 2.0 * math.pi, size=count)
    w = np.minimum(st["w"].uniform(0.0, 1.0, size=(count, 3)), _W_MAX)
    w_r = np.arctanh(w)
    if activated:
        planes = frame + [lam, a, k, w[:, 0], w[:, 1], w[:, 2]]
    else:
        planes = frame + [lam_r, a_r, k_r, w_r[:, 0], w_r[:, 1], w_r[:, 2]]
    return np.stack(planes).astype(np.float32), phase.astype(np.float32)


# Stored per-lobe scalars after the frame planes, per lobe family: the NASGabor
# lobe, NASG (no carrier frequency), SG (no anisotropy, no carrier) and the
# NASGabor lobe with a per-lobe carrier phase.
VARIANT_FIELDS = {
    "nasgabor": ("lam", "a", "k", "w0", "w1", "w2"),
    "nasg": ("lam", "a", "w0", "w1", "w2"),
    "sg": ("lam", "w0", "w1", "w2"),
    "phase": ("lam", "a", "k", "phi", "w0", "w1", "w2"),
}


def variant_planes(params: np.ndarray, phase, frame_mode: str, variant: str) -> np.ndarray:
    """Re-pack NASGabor planes [F + 6][N*L] for a lobe family: keep the frame planes
    and the family's fields in VARIANT_FIELDS order; the phase plane is `phase`."""
    f = 4 if frame_mode == FRAME_QUAT else 3
    src = {"lam": params[f], "a": params[f + 1], "k": params[f + 2], "w0": params[f + 3], "w1": params[f + 4],
           "w2": params[f + 5]}
    if variant == "phase":
        src["phi"] = np.asarray(phase, dtype=params.dtype)
    rows = [params[j] for j in range(f)] + [src[name] for name in VARIANT_FIELDS[variant]]
    return np.ascontiguousarray(np.stack(rows))


def variant_workload(n: int, n_lobes: int, seed: int, variant: str, frame_mode: str = FRAME_QUAT,
                     activated: bool = False) -> "Workload":
    """The point-cloud workload with its lobes stored for `variant` (the phase family
    stores the workload's phase draws, U[0, 2 pi])."""
    w = point_cloud_workload(n, n_lobes, seed, frame_mode, activated=activated)
    w.params = variant_planes(w.params, w.phase, frame_mode, variant)
    return w


def point_cloud_workload(n: int, n_lobes: int, seed: int, frame_mode: str = FRAME_QUAT,
                         with_upstream: bool = True, activated: bool = False) -> Workload:
    """Primitives uniform in the unit cube seen from one camera at (0, 0, 3).

    This is the small parity workload (N=4096, L=4) and the single-scene
    throughput workload (N=1e6, L=8): lobe parameters as in the module
    docstring, c0 ~ U[0, 1]^3, upstream dL/dRGB ~ N(0, 1).
    """
    st = _streams(seed)
    means = st["positions"].uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)
    params, phase = _draw_lobes(st, n * n_lobes, frame_mode, activated=activated)
    c0 = st["c0"].uniform(0.0, 1.0, size=(3, n)).astype(np.float32)
    g_rgb = st["upstream"].standard_normal((n, 3)).astype(np.float32) if with_upstream else None
    cam = np.array([0.0, 0.0, 3.0], dtype=np.float32)
    return Workload(n, n_lobes, frame_mode, params, c0, means, cam, g_rgb, phase)


def sh_coefficients(n: int, degree: int, seed: int) -> np.ndarray:
    """SH coefficients [(degree+1)^2][3][N] ~ N(0, 0.3^2) on the upstream substream's sibling."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5E]))
    nb = (degree + 1) ** 2
    return (0.3 * rng.standard_normal((nb, 3, n))).astype(np.float32)


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even) -> uint16 bit patterns."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    nan = np.isnan(x)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    out = rounded.astype(np.uint16)
    out[nan] = 0x7FC0
    return out


def from_bf16_bits(bits: np.ndarray) -> np.ndarray:
    """Exact widening of bfloat16 bit patterns to float32."""
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def quantize_bf16(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 (RNE) -> float32: the values a BF16-stored parameter holds."""
    return from_bf16_bits(to_bf16_bits(x))


# ---------------------------------------------------------------------------
# Scene-scale workload: noisy sphere shell seen by a ring of cameras.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class RingCamera:
    center: np.ndarray   # (3,) float32
    rot: np.ndarray      # (3, 3) float32 world->camera rows (right, up, forward)
    tan_half_fov: float


def _look_at(center: np.ndarray, target: np.ndarray, up: np.ndarray) -> np.ndarray:
    f = target - center
    f = f / np.linalg.norm(f)
    r = np.cross(f, up)
    r = r / np.linalg.norm(r)
    u = np.cross(r, f)
    return np.stack([r, u, f])


def _visible_fraction(means64: np.ndarray, cam: RingCamera) -> float:
    pc = (means64 - cam.center) @ cam.rot.T.astype(np.float64)
    z = pc[:, 2]
    t = cam.tan_half_fov
    vis = (z > 0) & (np.abs(pc[:, 0]) <= t * z) & (np.abs(pc[:, 1]) <= t * z)
    return float(vis.mean())


@dataclasses.dataclass
class ShellScene:
    n: int
    n_lobes: int
    frame_mode: str
    params: np.ndarray      # (P, N*L) float32 master copy
    c0: np.ndarray          # (3, N) float32
    means: np.ndarray       # (N, 3) float32
    cameras: list


def morton_order(points: np.ndarray, bits: int = 10) -> np.ndarray:
    """Permutation that sorts points by the Morton (Z-order) code of their
    coordinates quantised to `bits` bits per axis over their bounding box."""
    p = np.asarray(points, dtype=np.float64)
    lo = p.min(axis=0)
    span = np.maximum(p.max(axis=0) - lo, 1e-30)
    q = np.minimum(((p - lo) / span * (1 << bits)).astype(np.int64), (1 << bits) - 1)
    code = np.zeros(len(p), dtype=np.int64)
    for b in range(bits):
        for axis in range(3):
            code |= ((q[:, axis] >> b) & 1) << (3 * b + axis)
    return np.argsort(code, kind="stable")


def shell_scene(n: int, n_lobes: int, seed: int, n_cams: int = 8, ring_radius: float = 4.0,
                target_visible: float = 0.45, frame_mode: str = FRAME_QUAT,
                fov_sample: int = 200_000, order: str = "random") -> ShellScene:
    """Gaussians on a noisy sphere shell (radius U[1, 2]) and a ring of pinhole cameras.

    Cameras sit on the z=0 circle of radius `ring_radius` at angles 2*pi*j/n_cams,
    look at the origin with +z up, and share one symmetric field of view chosen
    by bisection so that camera 0 sees `target_visible` of the primitives
    (measured on a seeded subsample of `fov_sample` primitives). order="morton"
    stores the primitives in Morton order of their centres (same values).
    """
    st = _streams(seed)
    dirs = st["positions"].standard_normal((n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    radius = st["positions"].uniform(1.0, 2.0, size=(n, 1))
    means = (dirs * radius).astype(np.float32)
    params, _ = _draw_lobes(st, n * n_lobes, frame_mode)
    c0 = st["c0"].uniform(0.0, 1.0, size=(3, n)).astype(np.float32)
    up = np.array([0.0, 0.0, 1.0])
    cams = []
    for j in range(n_cams):
        ang = 2.0 * math.pi * j / n_cams
        c = np.array([ring_radius * math.cos(ang), ring_radius * math.sin(ang), 0.0])
        cams.append((c, _look_at(c, np.zeros(3), up)))
    sample = means[: min(n, fov_sample)].astype(np.float64)
    lo, hi = 1e-3, 10.0
    c_0, r_0 = cams[0]
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        frac = _visible_fraction(sample, RingCamera(c_0, r_0, mid))
        if frac < target_visible:
            lo = mid
        else:
            hi = mid
    t = float(np.float32(0.5 * (lo + hi)))
    cameras = [RingCamera(c.astype(np.float32), r.astype(np.float32), t) for c, r in cams]
    if order == "morton":
        # spatially coherent storage order (a layout choice: the primitives and
        # their values are the same, permuted together)
        perm = morton_order(means)
        means = np.ascontiguousarray(means[perm])
        c0 = np.ascontiguousarray(c0[:, perm])
        params = np.ascontiguousarray(
            params.reshape(params.shape[0], n, n_lobes)[:, perm, :].reshape(params.shape[0], -1))
    elif order != "random":
        raise ValueError(order)
    return ShellScene(n, n_lobes, frame_mode, params, c0, means, cameras)


def ring_upstream(n: int, cam_index: int, seed: int) -> np.ndarray:
    """Per-camera upstream dL/dRGB ~ N(0, 1), (N, 3) float32."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xC0, cam_index]))
    return rng.standard_normal((n, 3)).astype(np.float32)


# ---------------------------------------------------------------------------
# Batched workload: many independent scenes of uneven size.
# ---------------------------------------------------------------------------

def batched_scene_sizes(n_scenes: int, seed: int, n_min: int = 50_000, n_max: int = 3_000_000,
                        lobe_choices=(4, 8, 16)) -> list[tuple[int, int]]:
    """(N_s, L_s) per scene: N log-uniform in [n_min, n_max], L uniform over lobe_choices."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xBA7C]))
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_scenes)).astype(np.int64)
    ls = rng.choice(np.asarray(lobe_choices), size=n_scenes)
    return [(int(a), int(b)) for a, b in zip(ns, ls)]


# ---------------------------------------------------------------------------
# Fitting workload: a K=4 FP32 teacher field and a K=16 student.
# ---------------------------------------------------------------------------

# Learning-rate schedule of the fitting workload (constants only; the factor itself is
# the library's nasg_cosine_lr_factor and the oracle's schedule.cosine_factor): base
# rate 1e-3, 200 steps, the cosine schedule starting at iteration 47 = 200 x 7k/30k, the
# fraction of the optimisation after which the paper starts it (Supp. C). Step s (1-based)
# is iteration s - 1.
FIT_LR = 1e-3
FIT_STEPS = 200
FIT_SCHEDULE_START = 47


def fit_directions(step: int, seed: int, n_dirs: int = 64) -> np.ndarray:
    """View directions uniform on S^2 for one fitting step, (n_dirs, 3) float32 (unit up to fp32 rounding)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xD1, step]))
    d = rng.standard_normal((n_dirs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d.astype(np.float32)


def fit_subsample(n: int = 2_000_000, n_student: int = 16, n_teacher: int = 4, seed_teacher: int = 1005,
                  seed_student: int = 1006, sample: int = 20_000, seed_sample: int = 7):
    """The fitting workload's seeded subsample: teacher planes/c0, student planes/c0 (raw
    float32, both drawn over all n primitives) restricted to subsample_indices(n, sample,
    seed_sample), and those indices. Primitives are independent in the fit, so a fit of
    the subsample follows the same trajectories as those primitives inside the full run."""
    t = point_cloud_workload(n, n_teacher, seed_teacher, with_upstream=False)
    s = point_cloud_workload(n, n_student, seed_student, with_upstream=False)
    idx = subsample_indices(n, sample, seed_sample)
    lt = (idx[:, None] * n_teacher + np.arange(n_teacher)).reshape(-1)
    ls = (idx[:, None] * n_student + np.arange(n_student)).reshape(-1)
    return (np.ascontiguousarray(t.params[:, lt]), np.ascontiguousarray(t.c0[:, idx]),
            np.ascontiguousarray(s.params[:, ls]), np.ascontiguousarray(s.c0[:, idx]), idx)


def subsample_indices(n: int, count: int, seed: int) -> np.ndarray:
    """Sorted seeded subsample of primitive indices (int64)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5AB]))
    return np.sort(rng.choice(n, size=min(count, n), replace=False))


# ---------------------------------------------------------------------------
# On-device generation for the large throughput workloads (same distributions,
# drawn with torch's seeded generator on the GPU instead of numpy on the host).
# ---------------------------------------------------------------------------

def device_point_cloud(n: int, n_lobes: int, seed: int, device, param_dtype=None):
    """Point-cloud workload drawn on `device`: dict with params [P][N*L], c0 [3][N],
    means [N][3], g_rgb [N][3] (float32, params/c0 cast to param_dtype) and cam."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    count = n * n_lobes
    q = torch.randn((4, count), generator=g, device=device)
    q = q / q.norm(dim=0, keepdim=True)
    lam_r = torch.rand(count, generator=g, device=device) * math.log(1e3)
    a_r = torch.log(torch.rand(count, generator=g, device=device).clamp_min(_A_MIN))
    k = (torch.rand(count, generator=g, device=device) * 8.0).clamp_min(_K_MIN)
    k_r = torch.atanh(k / 20.0 - 1.0)
    w_r = torch.atanh(torch.rand((3, count), generator=g, device=device).clamp_max(_W_MAX))
    params = torch.cat([q, lam_r[None], a_r[None], k_r[None], w_r]).contiguous()
    c0 = torch.rand((3, n), generator=g, device=device)
    means = torch.rand((n, 3), generator=g, device=device)
    g_rgb = torch.randn((n, 3), generator=g, device=device)
    if param_dtype is not None:
        params = params.to(param_dtype)
        c0 = c0.to(param_dtype)
    return {"params": params, "c0": c0, "means": means, "g_rgb": g_rgb, "cam": (0.0, 0.0, 3.0), "n_lobes": n_lobes}
