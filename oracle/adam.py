"""FP64 CPU oracle for the optimiser update and the fused training steps.

TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the benchmark's
CPU-baseline leg; never by the product path. Shares no code with the CUDA path.

The paper builds on gsplat and says nothing of its optimiser beyond the
learning-rate heuristic (Sec. 4.2) and the cosine schedule (Supp. C); the
fused step follows Adam (Kingma & Ba) with bias correction, in the operation
order of torch.optim.Adam:
    m <- b1 m + (1 - b1) g ;  v <- b2 v + (1 - b2) g^2
    theta <- theta - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)
Parameters are stored as BF16 round-to-nearest-even copies of an FP32 master;
the model is evaluated at the BF16 values.

The fused step's upstream gradient is either given (dLoss/dRGB per primitive) or
that of a mean squared error against per-primitive target colours, the fit of
the appearance model (Sec. 4.2, eq:app_model) to colours: with the listed
primitives I (n_listed = |I|),
    Loss = (1 / (3 n_listed)) sum_{i in I} sum_c (c_ic - t_ic)^2,
    dLoss/dc_ic = 2 (c_ic - t_ic) / (3 n_listed).
"""
from __future__ import annotations

import numpy as np

from . import nasgabor as ng


def adam_update(theta, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step at step count t (>= 1). All arrays float64; returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    bc1 = 1.0 - beta1 ** t
    bc2 = 1.0 - beta2 ** t
    denom = np.sqrt(v) / np.sqrt(bc2) + eps
    theta = theta - (lr / bc1) * (m / denom)
    return theta, m, v


def bf16_round(x):
    """Round to bfloat16 (nearest even) through float32; returns float64 values."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def fused_step(master, m, v, c0_master, c0_m, c0_v, means, cam, g_rgb, idx, n_lobes, t,
               lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, frame_mode=ng.FRAME_QUAT,
               norm_mode=ng.NORM_APPROX, loss="given"):
    """Forward + backward + Adam for the primitives listed in idx (others untouched).

    master/m/v: (P, N*L); c0_master/c0_m/c0_v: (3, N); g_rgb: (N, 3) upstream
    gradient for every primitive (loss "given"), or the target colours (loss
    "mse": the mean squared error of the module docstring); only rows in idx are
    used. The model is evaluated at bf16_round(master). Returns dict with rgb
    (len(idx), 3), the upstream gradient used (g_rgb, len(idx) x 3), the loss
    (mse only) and the updated state arrays (float64, full size).
    """
    idx = np.asarray(idx, dtype=np.int64)
    P = ng.lobe_planes(frame_mode)
    n = np.asarray(means).shape[0]
    L = n_lobes
    lobe_idx = (idx[:, None] * L + np.arange(L)[None, :]).reshape(-1)
    p_sub = bf16_round(np.asarray(master, dtype=np.float64)[:, lobe_idx])
    c0_sub = bf16_round(np.asarray(c0_master, dtype=np.float64)[:, idx])
    mu = np.asarray(means)[idx]
    rgb = ng.forward(p_sub, c0_sub, mu, cam, L, frame_mode, norm_mode)
    value = None
    if loss == "given":
        g = np.asarray(g_rgb, dtype=np.float64)[idx]
    elif loss == "mse":
        res = rgb - np.asarray(g_rgb, dtype=np.float64)[idx]
        value = float(np.sum(res * res) / (3.0 * len(idx))) if len(idx) else 0.0
        g = 2.0 * res / (3.0 * max(len(idx), 1))
    else:
        raise ValueError(f"unknown loss {loss!r}")
    g_p, g_c0, _ = ng.backward(p_sub, c0_sub, mu, cam, g, L, frame_mode, norm_mode)
    out = {k: np.array(val, dtype=np.float64) for k, val in
           (("master", master), ("m", m), ("v", v), ("c0", c0_master), ("c0_m", c0_m), ("c0_v", c0_v))}
    th, mm, vv = adam_update(out["master"][:, lobe_idx], out["m"][:, lobe_idx], out["v"][:, lobe_idx],
                             g_p, t, lr, beta1, beta2, eps)
    out["master"][:, lobe_idx], out["m"][:, lobe_idx], out["v"][:, lobe_idx] = th, mm, vv
    th, mm, vv = adam_update(out["c0"][:, idx], out["c0_m"][:, idx], out["c0_v"][:, idx],
                             g_c0, t, lr, beta1, beta2, eps)
    out["c0"][:, idx], out["c0_m"][:, idx], out["c0_v"][:, idx] = th, mm, vv
    out["rgb"] = rgb
    out["g_rgb"] = g
    out["loss"] = value
    assert P == out["master"].shape[0]
    return out


def field_colours(params, c0, dirs, n_lobes, frame_mode=ng.FRAME_QUAT, norm_mode=ng.NORM_APPROX):
    """Colours (N, D, 3) of every primitive's lobe mixture at each of D shared directions."""
    params = np.asarray(params, dtype=np.float64)
    n = np.asarray(c0).shape[1]
    planes = ng.split_planes(params, n, n_lobes, frame_mode)
    act = ng.activate(planes, frame_mode)
    x, z = ng._frames(act, frame_mode)
    dirs = np.asarray(dirs, dtype=np.float64)
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    G = ng.lobe(dirs[None, :, None, :], x[:, None], z[:, None], act["lam"][:, None],
                act["a"][:, None], act["k"][:, None], norm_mode)          # (N, D, L)
    return np.asarray(c0, dtype=np.float64).T[:, None, :] + np.einsum("ndl,nlc->ndc", G, act["w"])


def fit_step(student, s_m, s_v, s_c0, s_c0_m, s_c0_v, teacher, t_c0, dirs, n_student, n_teacher, t,
             lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, frame_mode=ng.FRAME_QUAT,
             norm_mode=ng.NORM_APPROX, bf16_storage=True):
    """One fitting step of a student mixture to a teacher field at D shared directions.

    Per primitive the loss is the mean over (direction, channel) of the squared
    colour difference; the gradient of that per-primitive loss (summed over the
    directions) drives one Adam step of every primitive. Returns
    (new state dict, mse averaged over all primitives, directions and channels).
    """
    n = np.asarray(s_c0).shape[1]
    dirs = np.asarray(dirs, dtype=np.float64)
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    D = dirs.shape[0]
    sp = bf16_round(student) if bf16_storage else np.asarray(student, dtype=np.float64)
    sc0 = bf16_round(s_c0) if bf16_storage else np.asarray(s_c0, dtype=np.float64)
    target = field_colours(teacher, t_c0, dirs, n_teacher, frame_mode, norm_mode)
    planes = ng.split_planes(sp, n, n_student, frame_mode)
    act = ng.activate(planes, frame_mode)
    x, z = ng._frames(act, frame_mode)
    slope = ng.activation_slopes(act, ng.ACT_RAW)
    g_planes = np.zeros((ng.lobe_planes(frame_mode), n, n_student))
    g_c0 = np.zeros((3, n))
    sq = 0.0
    for j in range(D):
        dj = np.broadcast_to(dirs[j], (n, n_student, 3))
        G, par = ng.lobe(dj, x, z, act["lam"], act["a"], act["k"], norm_mode, need_grad=True)
        col = sc0.T + np.sum(act["w"] * G[..., None], axis=1)
        res = col - target[:, j, :]
        sq += np.sum(res * res)
        g_c = (2.0 / (3.0 * D)) * res                        # d(per-primitive mean)/dc
        g_c0 += g_c.T
        gG = np.sum(g_c[:, None, :] * act["w"], axis=-1)
        g_w = g_c[:, None, :] * G[..., None] * slope["w"]
        base = 4 if frame_mode == ng.FRAME_QUAT else 3
        g_planes[base + 0] += gG * par["lam"] * slope["lam"]
        g_planes[base + 1] += gG * par["a"] * slope["a"]
        g_planes[base + 2] += gG * par["k"] * slope["k"]
        for c in range(3):
            g_planes[base + 3 + c] += g_w[..., c]
        g_x = gG[..., None] * par["x"]
        g_z = gG[..., None] * par["z"]
        if frame_mode == ng.FRAME_QUAT:
            jx, jz = ng._quat_frame_jacobians(act["q"])
            g_q = np.einsum("nli,nlij->nlj", g_x, jx) + np.einsum("nli,nlij->nlj", g_z, jz)
            for c in range(4):
                g_planes[c] += g_q[..., c]
        else:
            raise NotImplementedError("the fitting workload uses QUAT frames")
    g_flat = g_planes.reshape(g_planes.shape[0], -1)
    new = {}
    new["student"], new["m"], new["v"] = adam_update(np.asarray(student, dtype=np.float64),
                                                     s_m, s_v, g_flat, t, lr, beta1, beta2, eps)
    new["c0"], new["c0_m"], new["c0_v"] = adam_update(np.asarray(s_c0, dtype=np.float64),
                                                      s_c0_m, s_c0_v, g_c0, t, lr, beta1, beta2, eps)
    return new, sq / (n * D * 3)
