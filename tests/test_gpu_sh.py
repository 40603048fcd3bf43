"""GPU parity of the real-SH comparison kernels (degree 0..3) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import sh as osh
from paper_2606_09794_gb300 import inputs
from tests._parity import colour_report, rel_l2, sensitivity_floor

pytestmark = pytest.mark.gpu


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
