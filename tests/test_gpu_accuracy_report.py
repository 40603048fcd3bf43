"""Error of the GPU path against the FP64 oracle, reported per output class and
precision on the parity workload (N = 4096, L = 4) and on a sampled slice of the
N = 1e6, L = 8 workload, through the fused forward+backward the benchmark times.
Prints one JSON line per case (run with -s to see it) and checks the bounds:
colours |dc| <= 1e-5 + 4 nu (FP32 parameters, and BF16 parameters against the
dequantised values), gradients relative L2 <= 1e-4 per plane. The BF16 storage
error (the oracle at the BF16 values against the oracle at the FP32 master
values) is reported and held to its first-order bound (tests/test_bf16_storage.py):
it is not within 4e-3 at these sharpnesses."""
import json

import numpy as np
import pytest

from oracle import nasgabor as ong
from paper_2606_09794_gb300 import inputs
from tests._parity import colour_report, rel_l2, sensitivity_floor
from tests.test_bf16_storage import storage_error_and_bound

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
    rep = colour_report(rgb.cpu().numpy()[idx], ref, nu, 1e-5)
    r_p, _, r_mu = ong.backward(pn, cn, mu, w.cam, g_np, L)
    gpn = gp.cpu().numpy()[:, lobes]
    planes = [rel_l2(gpn[k], r_p[k]) for k in range(gpn.shape[0])]
    out = {"n": int(len(idx)), "L": L, "params": "bf16" if bf16 else "f32", "colour": rep,
           "grad_rel_l2_max": max(planes), "grad_rel_l2_per_plane": [float(f"{x:.3g}") for x in planes],
           "g_means_rel_l2": rel_l2(gm.cpu().numpy()[idx], r_mu)}
    if bf16:
        q, bound, master = storage_error_and_bound(w, idx)
        out["bf16_storage_error"] = {"max_abs": float(q.max()),
                                     "max_rel1": float((q / np.maximum(1.0, np.abs(master))).max()),
                                     "max_over_first_order_bound": float((q / np.maximum(bound, 1e-300)).max())}
        assert np.all(q <= 1.5 * bound + 1e-9)
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
