"""Error of the GPU path against the FP64 oracle, reported per output class and
precision on the parity workload (N = 4096, L = 4) and on a sampled slice of the
N = 1e6, L = 8 workload, through the fused forward+backward the benchmark times.
Prints one JSON line per case (run with -s to see it) and checks the bounds:
colours |dc| <= base + 4 nu (base 1e-5 FP32, 4e-3 BF16 against the dequantised
values), gradients relative L2 <= 1e-4 per plane; the BF16 storage error
(BF16 parameters against the FP32 master values, both in the oracle) is reported."""
import json

import numpy as np
import pytest

from oracle import nasgabor as ong
from paper_2606_09794_gb300 import inputs
from tests._parity import colour_report, rel_l2, sensitivity_floor

pytestmark = pytest.mark.gpu


def _case(lib, w, bf16, sample=None):
    import torch
    p32 = torch.from_numpy(w.params).cuda()
    c32 = torch.from_numpy(w.c0).cuda()
    p, c = (p32.to(torch.bfloat16), c32.to(torch.bfloat16)) if bf16 else (p32, c32)
    means, g = torch.from_numpy(w.means).cuda(), torch.from_numpy(w.g_rgb).cuda()
    rgb, gp, gc0, gm = lib.nasgabor_fused_fwd_bwd(p, c, means, w.cam, g, w.n_lobes)
    torch.cuda.synchronize()
    L = w.n_lobes
    idx = np.arange(w.n) if sample is None else sample
    lobes = (idx[:, None] * L + np.arange(L)).reshape(-1)
    pn = inputs.quantize_bf16(w.params) if bf16 else w.params
    cn = inputs.quantize_bf16(w.c0) if bf16 else w.c0
    pn, cn = pn[:, lobes], cn[:, idx]
    mu, g_np = w.means[idx], w.g_rgb[idx]

    def fwd(p_, c_, m_, cam_):
        return ong.forward(p_, c_, m_, cam_, L)

    ref, nu = sensitivity_floor(fwd, (pn, cn, mu, w.cam), (0, 1, 2, 3))
    rep = colour_report(rgb.cpu().numpy()[idx], ref, nu, 4e-3 if bf16 else 1e-5)
    r_p, _, r_mu = ong.backward(pn, cn, mu, w.cam, g_np, L)
    gpn = gp.cpu().numpy()[:, lobes]
    planes = [rel_l2(gpn[k], r_p[k]) for k in range(gpn.shape[0])]
    out = {"n": int(len(idx)), "L": L, "params": "bf16" if bf16 else "f32", "colour": rep,
           "grad_rel_l2_max": max(planes), "grad_rel_l2_per_plane": [float(f"{x:.3g}") for x in planes],
           "g_means_rel_l2": rel_l2(gm.cpu().numpy()[idx], r_mu)}
    if bf16:
        master = ong.forward(w.params[:, lobes], w.c0[:, idx], mu, w.cam, L)
        q = np.abs(ref - master)
        out["bf16_storage_error"] = {"max_abs": float(q.max()),
                                     "max_rel1": float((q / np.maximum(1.0, np.abs(master))).max())}
    print(json.dumps(out))
    return out


@pytest.mark.parametrize("bf16", [False, True])
def test_accuracy_parity_workload(lib, bf16):
    out = _case(lib, inputs.point_cloud_workload(4096, 4, 1001), bf16)
    assert out["colour"]["violations"] == 0
    assert out["grad_rel_l2_max"] <= 1e-4 and out["g_means_rel_l2"] <= 1e-4


def test_accuracy_throughput_workload_sampled(lib):
    w = inputs.point_cloud_workload(1_000_000, 8, 1002)
    out = _case(lib, w, True, sample=inputs.subsample_indices(w.n, 3000, 11))
    assert out["colour"]["violations"] == 0
    assert out["grad_rel_l2_max"] <= 1e-4 and out["g_means_rel_l2"] <= 1e-4
