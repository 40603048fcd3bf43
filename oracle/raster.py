"""FP64 CPU oracle for the alpha-compositing consumer of the per-primitive colours.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.1 composites the primitives along a camera ray front to back:
    C(r) = sum_i T_i alpha_i c_i,   alpha_i = sigma_i rho_i,   T_i = prod_{j<i} (1 - alpha_j),
with rho_i the primitive's Gaussian kernel, projected approximately onto the image plane. The
readings used here (the paper delegates the projection and the compositing rules to the
3D Gaussian splatting rasterizer it builds on; each reading is listed in the design notes):

  P1 camera: p = R (mu - centre) with rows (right, up, forward); pixel coordinates
     x = cx + fx p_x / p_z, y = cy - fy p_y / p_z (y down); pixel (i, j) is sampled at its
     centre (i + 0.5, j + 0.5). Primitives with p_z <= near are not drawn.
  P2 projection: the local affine (EWA) approximation Sigma' = J R Sigma R^T J^T + b I, with
     Sigma = Rq diag(s^2) Rq^T (Sec. 3.1), J the Jacobian of (x, y) wrt p at the mean, and a
     screen-space low-pass b = 0.3 px^2; rho = exp(-q / 2), q = delta^T Sigma'^-1 delta,
     delta = pixel centre - projected mean.
  P3 alpha = min(0.99, sigma rho); a primitive contributes to a pixel iff alpha >= 1/255.
  P4 order: by p_z ascending, ties by primitive index.
  P5 early stop: before adding a contribution, if T (1 - alpha) < 1e-4 the pixel stops
     (that contribution and all later ones are dropped).
  P6 background 0; the pixel also reports its final transmittance T.

Backward (chain rule of the same sum; pinned by finite differences in the tests):
    dC/dc_i = alpha_i T_i,
    dC/dalpha_i = c_i T_i - (sum_{j > i, kept} c_j alpha_j T_j) / (1 - alpha_i),
    dalpha_i/dsigma_i = rho_i where alpha_i < 0.99 (0 where clamped).
"""
import numpy as np

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4
LOWPASS = 0.3


def quat_rotation(q):
    """Rotation matrices (N, 3, 3) of quaternions (w, x, y, z) (normalised here)."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], axis=-1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], axis=-1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], axis=-1),
    ], axis=-2)


def project(means, scales, quats, cam):
    """Per primitive: depth p_z, projected mean (x, y), Sigma' (2x2) and validity (P1, P2).

    cam: dict(rot (3x3), centre (3,), fx, fy, cx, cy, near)."""
    R = np.asarray(cam["rot"], dtype=np.float64)
    p = (np.asarray(means, dtype=np.float64) - np.asarray(cam["centre"], dtype=np.float64)) @ R.T
    z = p[:, 2]
    valid = z > cam["near"]
    zs = np.where(valid, z, 1.0)
    fx, fy = float(cam["fx"]), float(cam["fy"])
    x = cam["cx"] + fx * p[:, 0] / zs
    y = cam["cy"] - fy * p[:, 1] / zs
    J = np.zeros((p.shape[0], 2, 3))
    J[:, 0, 0] = fx / zs
    J[:, 0, 2] = -fx * p[:, 0] / (zs * zs)
    J[:, 1, 1] = -fy / zs
    J[:, 1, 2] = fy * p[:, 1] / (zs * zs)
    Rq = quat_rotation(quats)
    s2 = np.asarray(scales, dtype=np.float64) ** 2
    sigma3 = np.einsum("nij,nj,nkj->nik", Rq, s2, Rq)
    M = J @ R[None]
    sigma2 = M @ sigma3 @ np.transpose(M, (0, 2, 1)) + LOWPASS * np.eye(2)[None]
    return z, np.stack([x, y], axis=-1), sigma2, valid


def _alphas(px, py, mean2, sigma2, opacity):
    """alpha and rho of every primitive at one pixel centre (unclamped rho)."""
    d = np.stack([px - mean2[:, 0], py - mean2[:, 1]], axis=-1)
    a, b, c = sigma2[:, 0, 0], sigma2[:, 0, 1], sigma2[:, 1, 1]
    det = a * c - b * b
    q = (c * d[:, 0] ** 2 - 2 * b * d[:, 0] * d[:, 1] + a * d[:, 1] ** 2) / det
    rho = np.exp(-0.5 * q)
    return np.minimum(ALPHA_MAX, np.asarray(opacity, dtype=np.float64) * rho), rho


def render(means, scales, quats, opacity, colours, cam, width, height, pixels=None, with_margin=False):
    """Composite every pixel (or the listed (i, j) pixels). Returns image (H, W, 3) (or (K, 3)),
    final T, and with_margin the smallest relative distance of any decision to its threshold."""
    z, mean2, sigma2, valid = project(means, scales, quats, cam)
    order_all = np.lexsort((np.arange(len(z)), z))
    colours = np.asarray(colours, dtype=np.float64)
    if pixels is None:
        jj, ii = np.mgrid[0:height, 0:width]
        pixels = np.stack([ii.ravel(), jj.ravel()], axis=-1)
    out = np.zeros((len(pixels), 3))
    tfin = np.ones(len(pixels))
    margin = np.full(len(pixels), np.inf)
    for k, (i, j) in enumerate(pixels):
        alpha, _ = _alphas(i + 0.5, j + 0.5, mean2, sigma2, opacity)
        if np.any(valid):
            margin[k] = np.min(np.abs(alpha[valid] - ALPHA_MIN) / ALPHA_MIN)
        T = 1.0
        # the primitives that pass P1 and P3 at this pixel, in the P4 order
        for n in order_all[valid[order_all] & (alpha[order_all] >= ALPHA_MIN)]:
            a = alpha[n]
            test = T * (1.0 - a)
            margin[k] = min(margin[k], abs(test - T_MIN) / T_MIN)
            if test < T_MIN:
                break
            out[k] += colours[n] * a * T
            T = test
        tfin[k] = T
    if pixels is not None and out.shape[0] == width * height and len(pixels) == width * height:
        out = out.reshape(height, width, 3)
        tfin = tfin.reshape(height, width)
        margin = margin.reshape(height, width)
    return (out, tfin, margin) if with_margin else (out, tfin)


def render_backward(means, scales, quats, opacity, colours, cam, width, height, g_image):
    """Gradients of <g_image, image> wrt the colours (N, 3) and the opacities (N,)."""
    z, mean2, sigma2, valid = project(means, scales, quats, cam)
    order_all = np.lexsort((np.arange(len(z)), z))
    colours = np.asarray(colours, dtype=np.float64)
    opacity = np.asarray(opacity, dtype=np.float64)
    g_image = np.asarray(g_image, dtype=np.float64).reshape(height, width, 3)
    g_c = np.zeros_like(colours)
    g_o = np.zeros(len(z))
    for j in range(height):
        for i in range(width):
            alpha, rho = _alphas(i + 0.5, j + 0.5, mean2, sigma2, opacity)
            kept, T = [], 1.0
            for n in order_all[valid[order_all] & (alpha[order_all] >= ALPHA_MIN)]:
                test = T * (1.0 - alpha[n])
                if test < T_MIN:
                    break
                kept.append((n, alpha[n], T))
                T = test
            g = g_image[j, i]
            after = np.zeros(3)                     # sum_{later kept} c_j alpha_j T_j
            for n, a, Tn in reversed(kept):
                g_c[n] += g * a * Tn
                d_alpha = float(np.dot(g, colours[n] * Tn - after / (1.0 - a)))
                if opacity[n] * rho[n] < ALPHA_MAX:
                    g_o[n] += d_alpha * rho[n]
                after += colours[n] * a * Tn
    return g_c, g_o


def footprint_radius(sigma2, opacity):
    """Half-width of a square that holds every pixel centre where alpha >= 1/255:
    q <= 2 ln(255 sigma) and |delta|^2 <= lambda_max q. -1 where the primitive can never reach 1/255."""
    a, b, c = sigma2[:, 0, 0], sigma2[:, 0, 1], sigma2[:, 1, 1]
    lmax = 0.5 * (a + c) + np.sqrt(0.25 * (a - c) ** 2 + b * b)
    lnr = np.log(np.maximum(255.0 * np.asarray(opacity, dtype=np.float64), 1e-300))
    return np.where(lnr > 0, np.sqrt(lmax * 2.0 * np.maximum(lnr, 0.0)), -1.0)


def camera(rot, centre, width, height, tan_half_fov_x, near=0.2):
    """Pinhole camera dict with square pixels from a horizontal half-FOV tangent."""
    fx = 0.5 * width / tan_half_fov_x
    return {"rot": np.asarray(rot, dtype=np.float64), "centre": np.asarray(centre, dtype=np.float64),
            "fx": fx, "fy": fx, "cx": 0.5 * width, "cy": 0.5 * height, "near": float(near)}
