"""GPU parity of the real-SH comparison kernels (degree 0..3) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import sh as osh
from paper_2606_09794_gb300 import inputs
from tests._parity import colour_report, grad_report, rel_l2, sensitivity_floor

pytestmark = pytest.mark.gpu


def _grad_elementwise(gc, gm, coeffs, means, cam, g, degree):
    """Every gradient element against the oracle: |dg| <= 1e-4 |g| + 4 nu + f, f for the
    means the FP32 rounding floor of dLoss/dd = sum_j (dLoss/dY_j) grad Y_j projected by
    I - d d^T: the kernel differentiates the basis polynomials in Cartesian form, whose
    gradient adds to the tangent one a radial part of about l Y_j for a degree-l term, so
    f = 16 x 2^-24 x (the terms' magnitudes + their radial parts along d_c) / |mu - cam|."""
    def bwd(c, m, cm):
        r_c, r_m = osh.backward(c, m, cm, g, degree)
        return np.concatenate([r_c.ravel(), r_m.ravel()])

    ref, nu = sensitivity_floor(bwd, (coeffs, means, cam), (0, 1, 2))
    r = np.asarray(means, np.float64) - np.asarray(cam, np.float64)
    dist = np.linalg.norm(r, axis=-1)
    d = r / dist[:, None]
    Y, gY = osh.basis(d, degree, need_grad=True)
    wj = np.abs(np.einsum("jcn,nc->nj", np.asarray(coeffs, np.float64), np.asarray(g, np.float64)))
    terms = np.einsum("nj,njk->nk", wj, np.abs(gY))
    ls = np.floor(np.sqrt(np.arange(Y.shape[-1])))                 # degree of basis function j
    radial = np.sum(wj * ls * np.abs(Y), axis=-1, keepdims=True)
    fm = 16 * 2.0 ** -24 * (terms + (np.linalg.norm(terms, axis=-1, keepdims=True) + radial) * np.abs(d)) / dist[:, None]
    nc = np.asarray(coeffs).size
    atol = np.concatenate([np.full(nc, 1e-12 * np.abs(ref[:nc]).max()), fm.ravel() + 1e-12 * np.abs(ref[nc:]).max()])
    got = np.concatenate([np.asarray(gc, np.float64).ravel(), np.asarray(gm, np.float64).ravel()])
    return grad_report(got, ref, nu, atol=atol)


@pytest.mark.parametrize("degree,n", [(0, 100), (1, 257), (2, 1000), (3, 4099), (3, 1)])
def test_sh_parity(lib, degree, n):
    import torch
    rng = np.random.default_rng(degree * 100 + n)
    means = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    cam = np.array([0.0, 0.0, 3.0], np.float32)
    coeffs = inputs.sh_coefficients(n, degree, 5)
    g = rng.standard_normal((n, 3)).astype(np.float32)
    c_d = torch.from_numpy(coeffs).cuda()
    m_d = torch.from_numpy(means).cuda()
    rgb = lib.sh_eval_fwd(c_d, m_d, cam, degree)
    gc, gm = lib.sh_eval_bwd(c_d, m_d, cam, torch.from_numpy(g).cuda(), degree)
    torch.cuda.synchronize()

    def fwd(c, m, cm):
        return osh.forward(c, m, cm, degree)

    ref, nu = sensitivity_floor(fwd, (coeffs, means, cam), (0, 1, 2))
    rep = colour_report(rgb.cpu().numpy(), ref, nu, 1e-5)
    assert rep["violations"] == 0, rep
    r_c, r_m = osh.backward(coeffs, means, cam, g, degree)
    assert rel_l2(gc.cpu().numpy(), r_c) <= 1e-6
    if degree > 0:
        assert rel_l2(gm.cpu().numpy(), r_m) <= 1e-4
    else:
        assert np.abs(gm.cpu().numpy()).max() < 1e-6
    rep = _grad_elementwise(gc.cpu().numpy(), gm.cpu().numpy(), coeffs, means, cam, g, degree)
    assert rep["violations"] == 0, rep


def test_sh_full_size_sampled(lib):
    import torch
    n = 1_000_000
    w = inputs.point_cloud_workload(n, 1, 1002)
    coeffs = inputs.sh_coefficients(n, 3, 1002)
    sample = inputs.subsample_indices(n, 20_000, 2)
    c_d = torch.from_numpy(coeffs).cuda()
    m_d = torch.from_numpy(w.means).cuda()
    g_d = torch.from_numpy(w.g_rgb).cuda()
    rgb = lib.sh_eval_fwd(c_d, m_d, w.cam)
    gc, gm = lib.sh_eval_bwd(c_d, m_d, w.cam, g_d)
    torch.cuda.synchronize()
    cs = coeffs[:, :, sample]
    ref, nu = sensitivity_floor(lambda c, m, cm: osh.forward(c, m, cm), (cs, w.means[sample], w.cam), (0, 1, 2))
    rep = colour_report(rgb.cpu().numpy()[sample], ref, nu, 1e-5)
    assert rep["violations"] == 0, rep
    r_c, r_m = osh.backward(cs, w.means[sample], w.cam, w.g_rgb[sample])
    assert rel_l2(gc.cpu().numpy()[:, :, sample], r_c) <= 1e-6
    assert rel_l2(gm.cpu().numpy()[sample], r_m) <= 1e-4
    rep = _grad_elementwise(gc.cpu().numpy()[:, :, sample], gm.cpu().numpy()[sample], cs, w.means[sample], w.cam,
                            w.g_rgb[sample], 3)
    assert rep["violations"] == 0, rep


def test_sh_autograd(lib):
    import torch
    n = 500
    rng = np.random.default_rng(4)
    coeffs = torch.from_numpy(inputs.sh_coefficients(n, 3, 4)).cuda().requires_grad_(True)
    means = torch.from_numpy(rng.uniform(0, 1, (n, 3)).astype(np.float32)).cuda().requires_grad_(True)
    g = torch.randn(n, 3, device="cuda")
    out = lib.ShEval.apply(coeffs, means, (0.0, 0.0, 3.0), 3)
    out.backward(g)
    gc, gm = lib.sh_eval_bwd(coeffs.detach(), means.detach(), (0, 0, 3), g)
    torch.testing.assert_close(coeffs.grad, gc, rtol=0, atol=0)
    torch.testing.assert_close(means.grad, gm, rtol=0, atol=0)
