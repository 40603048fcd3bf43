"""The library's FP32 elementary functions (expm1, tanh with 1 - tanh^2, sincos)
against float64 numpy, in units of the float32 spacing of the true value."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ulp_err(got, ref):
    ref32 = ref.astype(np.float32)
    spacing = np.spacing(np.abs(ref32)).astype(np.float64)
    spacing = np.maximum(spacing, np.float64(np.finfo(np.float32).tiny))
    return np.abs(got.astype(np.float64) - ref) / spacing


def _run(lib, fn, x):
    import torch
    y, y2 = lib.nasg_math_probe(fn, torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    return y.cpu().numpy(), None if y2 is None else y2.cpu().numpy()


def test_expm1(lib):
    """e^x - 1 on x <= 0, the kernels' only use (arguments (1+tau) ln kappa and -2 lam)."""
    rng = np.random.default_rng(1)
    x = -np.concatenate([rng.uniform(0, 1, 200000), rng.uniform(0, 200, 200000),
                         10.0 ** rng.uniform(-30, 0, 100000), [0.0, 0.5, 0.49999997, 0.50000006]])
    x = x.astype(np.float32)
    y, _ = _run(lib, 0, x)
    ref = np.expm1(x.astype(np.float64))
    err = _ulp_err(y, ref)
    assert err.max() <= 8.0, (err.max(), x[np.argmax(err)])


def test_tanh_and_sech2(lib):
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-1, 1, 200000), rng.uniform(-30, 30, 200000),
                        np.sign(rng.standard_normal(100000)) * 10.0 ** rng.uniform(-30, 0, 100000),
                        [0.0, 0.25, -0.25, 50.0, -50.0]]).astype(np.float32)
    t, s = _run(lib, 1, x)
    x64 = x.astype(np.float64)
    assert _ulp_err(t, np.tanh(x64)).max() <= 8.0
    sech2 = 1.0 / np.cosh(np.minimum(np.abs(x64), 300)) ** 2
    # relative where representable; absolute 1e-37 below the normal range
    # e^{-2|x|} comes from 2^(-2|x| log2 e): the rounding of the argument adds ~|x| 1.2e-7
    rel = np.abs(s - sech2) / np.maximum(sech2, 1e-30)
    bound = 6e-7 + 1.2e-7 * np.abs(x64)
    keep = sech2 > 1e-30
    assert (rel[keep] <= bound[keep]).all()


def test_tanh_table_matches_evaluation_bitwise(lib):
    """The BF16 kernels' weight table against the evaluation at every finite BF16 value,
    both signs: tanh bit for bit everywhere (the table's range and the closed forms on
    either side of it); 1 - tanh^2 bit for bit from 2^-13 on, and below it the closed
    form 1 - x^2, within 8 ulps of the evaluation and exact to rounding."""
    bits = np.arange(0, 0x7f80, dtype=np.uint32)             # every finite BF16 magnitude
    bits = np.concatenate([bits, bits | 0x8000])
    x = (bits << 16).view(np.float32)
    t_eval, s_eval = _run(lib, 1, x)
    t_tab, s_tab = _run(lib, 3, x)
    assert np.array_equal(t_eval.view(np.uint32), t_tab.view(np.uint32))
    big = np.abs(x) >= 2.0 ** -13
    assert np.array_equal(s_eval[big].view(np.uint32), s_tab[big].view(np.uint32))
    x64 = x[~big].astype(np.float64)
    assert np.array_equal(s_tab[~big], (1.0 - x64 * x64).astype(np.float32))
    assert _ulp_err(s_eval[~big], 1.0 - x64 * x64).max() <= 8.0


def test_sincos(lib):
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-4, 4, 200000), rng.uniform(-25, 25, 200000),
                        rng.uniform(-6400, 6400, 50000), 10.0 ** rng.uniform(-30, 0, 50000),
                        np.arange(-16, 17) * (np.pi / 2)]).astype(np.float32)
    s, c = _run(lib, 2, x)
    x64 = x.astype(np.float64)
    # absolute error for |x| <= 25 (the kernels' range: |k v / 2| <= 20)
    small = np.abs(x64) <= 25
    assert np.abs(s - np.sin(x64))[small].max() <= 1.5e-7
    assert np.abs(c - np.cos(x64))[small].max() <= 1.5e-7
    assert np.abs(s - np.sin(x64)).max() <= 2e-6
    assert np.abs(c - np.cos(x64)).max() <= 2e-6


def test_pipe_probe_rates(lib):
    """The pipe microbenchmark gives issue rates within the nominal range of a 152-SM part
    at up to 2.07 GHz: MUFU ex2 results (16 or 32 per clock per SM: 5e12..1.1e13/s), FP32
    FMA lane-instructions (128 per clock per SM: at most 4.0e13/s), packed pairs counting
    two operations, and each rate reproducible (two measurements within 5 %)."""
    r0, r0b = lib.nasg_pipe_rate(0), lib.nasg_pipe_rate(0)
    r1 = lib.nasg_pipe_rate(1)
    r2 = lib.nasg_pipe_rate(2)
    assert 1e12 < r0 < 2e13 and abs(r0 - r0b) <= 0.05 * r0, (r0, r0b)
    assert 5e12 < r2 < 5e13, r2
    assert 5e12 < r1 < 1e14, r1
    print({"mufu_ex2_per_s": r0, "ffma2_ops_per_s": r1, "ffma_per_s": r2})
