"""Spherical quadrature used by the oracle pins (tests only).

Integrates a function of the direction over S^2 in a local frame whose pole is
the lobe axis z = e_z and whose tangent x = e_x: d = (sqrt(1-u^2) cos phi,
sqrt(1-u^2) sin phi, u). The u integral is composite Gauss-Legendre, the phi integral is
the trapezoidal rule, which is spectrally accurate for periodic integrands.
The u intervals are refined geometrically toward both poles.
"""
import numpy as np


def sphere_grid(n_phi=512, n_gl=48, n_intervals=36, t_min=1e-9):
    xg, wg = np.polynomial.legendre.leggauss(n_gl)
    # breakpoints in u refined geometrically toward both poles: toward u = 1 for
    # sharp lobes, toward u = -1 where kappa^tau has an endpoint singularity
    t = np.geomspace(1.0, t_min, n_intervals)
    br = np.unique(np.concatenate([[-1.0, 1.0], 1.0 - t, -1.0 + t]))
    us, wus = [], []
    for a, b in zip(br[:-1], br[1:]):
        us.append(0.5 * (b - a) * xg + 0.5 * (b + a))
        wus.append(0.5 * (b - a) * wg)
    u = np.concatenate(us)
    wu = np.concatenate(wus)
    phi = np.arange(n_phi) * (2.0 * np.pi / n_phi)
    wphi = np.full(n_phi, 2.0 * np.pi / n_phi)
    U, PHI = np.meshgrid(u, phi, indexing="ij")
    W = wu[:, None] * wphi[None, :]
    s = np.sqrt(np.maximum(0.0, 1.0 - U * U))
    d = np.stack([s * np.cos(PHI), s * np.sin(PHI), U], axis=-1).reshape(-1, 3)
    return d, W.reshape(-1)


def integrate_lobe(lobe_fn, lam, a, k, norm_mode, **grid_kw):
    """int_{S^2} G(d; [e_x, e_y, e_z], lam, a, k) d omega by quadrature."""
    d, w = sphere_grid(**grid_kw)
    x = np.broadcast_to(np.array([1.0, 0.0, 0.0]), d.shape)
    z = np.broadcast_to(np.array([0.0, 0.0, 1.0]), d.shape)
    n = d.shape[0]
    g = lobe_fn(d, x, z, np.full(n, float(lam)), np.full(n, float(a)), np.full(n, float(k)), norm_mode)
    return float(np.sum(g * w))
