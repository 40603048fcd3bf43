"""GPU parity of the compositing consumer (nasg_raster_forward / _backward) against
the FP64 oracle (oracle/raster.py). Pixels whose alpha or transmittance decision
lies within 1e-4 (relative) of its threshold may legitimately differ between FP32
and FP64; they are excluded (and their upstream gradient set to 0) and must stay rare."""
import numpy as np
import pytest

from oracle import nasgabor as ong
from oracle import raster as orr
from paper_2606_09794_gb300 import inputs
from tests._parity import rel_l2

pytestmark = pytest.mark.gpu

MARGIN = 1e-4


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _scene(n, seed, spread=1.0, log_scale=(-3.0, -1.6), centre=(0.0, 0.0, 0.0)):
    rng = np.random.default_rng(seed)
    means = (np.asarray(centre) + rng.uniform(-spread, spread, (n, 3))).astype(np.float32)
    scales = np.exp(rng.uniform(*log_scale, (n, 3))).astype(np.float32)
    quats = rng.normal(size=(n, 4)).astype(np.float32)
    opacity = rng.uniform(0.02, 0.98, n).astype(np.float32)
    colours = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    return means, scales, quats, opacity, colours


def _cams(lib, width, height, tan=0.4, centre=(0.0, 0.0, -4.0), yaw=0.0):
    c, s = np.cos(yaw), np.sin(yaw)
    rot = np.array([[c, 0, -s], [0, 1, 0], [s, 0, c]])
    fx = 0.5 * width / tan
    cam = lib.raster_camera(rot, centre, width, height, fx)
    ocam = {"rot": rot, "centre": np.asarray(centre, np.float64), "fx": np.float32(fx), "fy": np.float32(fx),
            "cx": 0.5 * width, "cy": 0.5 * height, "near": np.float32(0.2)}
    return cam, ocam


def _run(lib, sc, cam, max_pairs=1 << 22):
    r = lib.Raster(len(sc[0]), cam, max_pairs)
    img, T = r.forward(*[_dev(x) for x in sc])
    return r, img, T


@pytest.mark.parametrize("w,h,n,seed,log_scale", [(64, 48, 300, 1, (-3.0, -1.6)), (37, 29, 150, 2, (-2.5, -1.5)),
                                                  (48, 32, 2500, 3, (-3.5, -2.0))])
def test_forward_matches_oracle(lib, w, h, n, seed, log_scale):
    import torch
    sc = _scene(n, seed, log_scale=log_scale)
    cam, ocam = _cams(lib, w, h)
    _, img, T = _run(lib, sc, cam)
    torch.cuda.synchronize()
    ref, tref, margin = orr.render(*sc, ocam, w, h, with_margin=True)
    ok = margin > MARGIN
    assert ok.mean() > 0.97, ok.mean()
    gi, gt = img.cpu().numpy(), T.cpu().numpy()
    assert np.abs(gi - ref)[ok].max() <= 5e-5, np.abs(gi - ref)[ok].max()
    assert np.abs(gt - tref)[ok].max() <= 5e-5
    # deterministic: a second forward gives the same bits
    _, img2, T2 = _run(lib, sc, cam)
    torch.testing.assert_close(img2, img, rtol=0, atol=0)


def test_backward_matches_oracle(lib):
    import torch
    w, h, n = 48, 36, 220
    sc = _scene(n, 11)
    cam, ocam = _cams(lib, w, h)
    r, img, T = _run(lib, sc, cam)
    _, _, margin = orr.render(*sc, ocam, w, h, with_margin=True)
    g = np.random.default_rng(12).normal(size=(h, w, 3))
    g[margin <= MARGIN] = 0.0
    gc, go = r.backward(_dev(sc[4]), T, _dev(g))
    torch.cuda.synchronize()
    rc, ro = orr.render_backward(*sc, ocam, w, h, g)
    assert rel_l2(gc.cpu().numpy(), rc) <= 1e-4
    assert rel_l2(go.cpu().numpy(), ro) <= 1e-4


def test_large_frame_sampled_pixels(lib):
    """1280 x 720, 200k primitives (many tiles with several 256-primitive batches):
    300 sampled pixels against the oracle."""
    import torch
    w, h, n = 1280, 720, 200_000
    sc = _scene(n, 21, spread=1.5, log_scale=(-5.0, -3.0))
    cam, ocam = _cams(lib, w, h, tan=0.6)
    r, img, T = _run(lib, sc, cam, max_pairs=1 << 24)
    assert r.n_pairs > n
    torch.cuda.synchronize()
    rng = np.random.default_rng(22)
    pix = np.stack([rng.integers(0, w, 300), rng.integers(0, h, 300)], axis=1)
    ref, tref, margin = orr.render(*sc, ocam, w, h, pixels=pix, with_margin=True)
    got = img.cpu().numpy()[pix[:, 1], pix[:, 0]]
    ok = margin > MARGIN
    assert ok.mean() > 0.9
    assert np.abs(got - ref)[ok].max() <= 1e-4


def test_edge_cases(lib):
    import torch
    cam, _ = _cams(lib, 40, 24)
    # no primitives
    r = lib.Raster(0, cam, 16)
    e = torch.empty((0, 3), device="cuda")
    img, T = r.forward(e, e, torch.empty((0, 4), device="cuda"), torch.empty(0, device="cuda"), e)
    assert float(img.abs().max()) == 0.0 and float(T.min()) == 1.0
    # everything behind the camera
    sc = list(_scene(50, 31, centre=(0.0, 0.0, -8.0)))
    r, img, T = _run(lib, sc, cam)
    assert float(img.abs().max()) == 0.0 and r.n_pairs == 0
    # pair capacity: reported, not overrun
    sc = _scene(400, 32)
    r = lib.Raster(400, cam, 8)
    with pytest.raises(lib.NasgError) as ei:
        r.forward(*[_dev(x) for x in sc])
    assert ei.value.status == -7


def test_real_colour_gradient_drives_the_appearance_backward(lib):
    """Chain: NASGabor colours at the camera -> composite -> loss against a target
    image -> dLoss/dcolour (real, from the compositing backward) -> NASGabor
    backward; the lobe-parameter gradients against the oracle's chain."""
    import torch
    w, h, n, L = 40, 30, 160, 4
    wl = inputs.point_cloud_workload(n, L, 41)
    rng = np.random.default_rng(42)
    means = (rng.uniform(-1, 1, (n, 3))).astype(np.float32)
    scales = np.exp(rng.uniform(-2.6, -1.6, (n, 3))).astype(np.float32)
    quats = rng.normal(size=(n, 4)).astype(np.float32)
    opacity = rng.uniform(0.1, 0.9, n).astype(np.float32)
    cam, ocam = _cams(lib, w, h)
    centre = ocam["centre"].astype(np.float32)
    params, c0 = _dev(wl.params), _dev(wl.c0)
    rgb = lib.nasgabor_eval_fwd(params, c0, _dev(means), tuple(centre), L)
    r = lib.Raster(n, cam, 1 << 20)
    img, T = r.forward(_dev(means), _dev(scales), _dev(quats), _dev(opacity), rgb)
    colours_ref = ong.forward(wl.params, wl.c0, means, centre, L)
    ref, tref, margin = orr.render(means, scales, quats, opacity, colours_ref, ocam, w, h, with_margin=True)
    target = rng.uniform(0, 1, (h, w, 3))
    g = 2.0 * (ref - target) / target.size
    g[margin <= MARGIN] = 0.0
    gc, _ = r.backward(rgb, T, _dev(g))
    gp, _, _ = lib.nasgabor_eval_bwd(params, _dev(means), tuple(centre), gc, L)
    torch.cuda.synchronize()
    rc, _ = orr.render_backward(means, scales, quats, opacity, colours_ref, ocam, w, h, g)
    assert rel_l2(gc.cpu().numpy(), rc) <= 2e-4
    rp, _, _ = ong.backward(wl.params, wl.c0, means, centre, rc, L)
    gpn = gp.cpu().numpy()
    assert max(rel_l2(gpn[p], rp[p]) for p in range(10)) <= 5e-4
