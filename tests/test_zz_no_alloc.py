"""The allocation-free compaction entry point (nasg_frustum_compact_noalloc),
for callers that cannot allocate device memory where they need the visible
list (a renderer inside a host application that owns every device allocation,
or a per-frame loop where a cudaMalloc would synchronise the device). Its
output must equal the workspace entry point's exactly (integer indices), on
consecutive calls that reuse the library's shared scratch. Kept in its own file,
collected last, so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2606_09794_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_compaction_matches_workspace_entry_point(lib):
    import torch
    # two calls in a row with different scenes and cameras (the second call's
    # list is shorter than the first's, so stale scratch would show)
    cases = [(inputs.shell_scene(300_000, 1, 501, fov_sample=50_000), 0),
             (inputs.shell_scene(70_001, 1, 502, fov_sample=50_000, target_visible=0.2), 3)]
    for sc, j in cases:
        cam = sc.cameras[j]
        means = torch.from_numpy(sc.means).cuda()
        ref_idx, ref_n = lib.nasg_frustum_compact(means, cam.rot, cam.center, cam.tan_half_fov)
        got_idx, got_n = lib.nasg_frustum_compact_noalloc(means, cam.rot, cam.center, cam.tan_half_fov)
        torch.cuda.synchronize()
        k = int(ref_n.item())
        assert int(got_n.item()) == k and k > 0
        np.testing.assert_array_equal(got_idx[:k].cpu().numpy(), ref_idx[:k].cpu().numpy())


def test_noalloc_rejects_problems_beyond_capacity(lib):
    import torch
    means = torch.zeros((4, 3), device="cuda")
    rot = (ctypes.c_float * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    cen = (ctypes.c_float * 3)(0, 0, 0)
    nv = torch.zeros(1, device="cuda", dtype=torch.int32)
    st = lib.lib.nasg_frustum_compact_noalloc(lib.NOALLOC_MAX_PRIMS + 1, ctypes.c_void_p(means.data_ptr()), rot, cen,
                                              0.5, 0.0, ctypes.c_void_p(nv.data_ptr()), ctypes.c_void_p(nv.data_ptr()),
                                              None)
    assert st == -7
