"""FP64 CPU oracle for the learning-rate rules of the method (test infrastructure only).

* Sec. 4.2 (learning-rate heuristic): with d_knn the mean, over cameras, of the
  mean distance from a camera centre to its k nearest other camera centres,
      eta_f     = eta_f_base     (d_ref / d_knn)^beta,
      eta_sigma = eta_sigma_base (d_knn / d_ref)^gamma,
  with beta = 2, gamma = 0.6, k = 3 in the paper. d_ref is the same quantity for
  a reference capture (a dataset-specific constant, passed in).
* Supp. (LR scheduling): eta(t) = (1 + cos(pi t / T_max)) / 2 multiplies the
  base rates once the schedule starts; here t and T_max count from the start of
  the schedule (t_start), and the factor is 1 before it.

Brute force: all pairwise distances, a full sort per camera.
"""
import math

import numpy as np


def knn_camera_distance(centres, k=3):
    """Mean over cameras of the mean distance to the k nearest other cameras
    (all others when there are fewer than k)."""
    c = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    n = c.shape[0]
    if n < 2:
        raise ValueError("need at least two cameras")
    kk = min(k, n - 1)
    per_cam = []
    for i in range(n):
        d = sorted(math.sqrt(float(np.sum((c[i] - c[j]) ** 2))) for j in range(n) if j != i)
        per_cam.append(sum(d[:kk]) / kk)
    return sum(per_cam) / n


def lr_heuristic(centres, d_ref, eta_f_base, eta_sigma_base, k=3, beta=2.0, gamma=0.6):
    """(eta_f, eta_sigma, d_knn) of the Sec. 4.2 heuristic."""
    d = knn_camera_distance(centres, k)
    return eta_f_base * (d_ref / d) ** beta, eta_sigma_base * (d / d_ref) ** gamma, d


def cosine_factor(t, t_max, t_start=0):
    """LR multiplier at iteration t: 1 before t_start, then (1 + cos(pi s / S)) / 2
    with s = t - t_start, S = t_max - t_start (0 from s >= S on)."""
    if t < t_start:
        return 1.0
    s, span = t - t_start, t_max - t_start
    if s >= span:
        return 0.0
    return 0.5 * (1.0 + math.cos(math.pi * s / span))
