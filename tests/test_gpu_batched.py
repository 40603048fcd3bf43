"""The batched persistent launch: every scene's outputs equal the single-scene fused
kernel's (same arithmetic, up to FMA contraction in a few scalar terms), oracle
parity on sampled scenes, replay from a captured CUDA graph, and the autotuner."""
import numpy as np
import pytest

from oracle import nasgabor as ong
from paper_2606_09794_gb300 import inputs
from tests._parity import chain_floor, colour_report, grad_report, rel_l2, sensitivity_floor

pytestmark = pytest.mark.gpu


def _scenes(sizes, seed, bf16, frame="quat"):
    import torch
    out = []
    for j, (n, L) in enumerate(sizes):
        w = inputs.point_cloud_workload(n, L, seed + j, frame)
        p = torch.from_numpy(w.params).cuda()
        c0 = torch.from_numpy(w.c0).cuda()
        if bf16:
            p, c0 = p.to(torch.bfloat16), c0.to(torch.bfloat16)
        cam = (0.1 * j, -0.05 * j, 3.0)
        out.append(dict(params=p, c0=c0, means=torch.from_numpy(w.means).cuda(), g_rgb=torch.from_numpy(w.g_rgb).cuda(),
                        cam=cam, n_lobes=L, w=w))
    return out


def _compare_with_single(lib, scenes, frame="quat", norm="approx"):
    import torch
    for sc in scenes:
        if sc["means"].shape[0] == 0:
            continue
        ref = lib.nasgabor_fused_fwd_bwd(sc["params"], sc["c0"], sc["means"], sc["cam"], sc["g_rgb"], sc["n_lobes"],
                                         frame_mode=frame, norm_mode=norm)
        torch.testing.assert_close(sc["rgb"], ref[0], rtol=1e-6, atol=1e-5)
        gp, rp = sc["g_params"].cpu().numpy(), ref[1].cpu().numpy()
        assert max(rel_l2(gp[p], rp[p]) for p in range(gp.shape[0])) < 1e-5
        torch.testing.assert_close(sc["g_c0"], ref[2], rtol=0, atol=0)
        assert rel_l2(sc["g_means"].cpu().numpy(), ref[3].cpu().numpy()) < 1e-5


SIZES = [(5000, 8), (1, 4), (777, 16), (12345, 4), (0, 8), (4099, 3), (2048, 8), (301, 1)]


@pytest.mark.parametrize("bf16", [True, False])
@pytest.mark.parametrize("dynamic,sub_tiles,staged", [(1, 1, 0), (0, 3, 0), (1, 8, 0), (1, 1, 1), (0, 3, 1),
                                                      (1, 4, 1)])
def test_batched_equals_single_scene_kernel(lib, bf16, dynamic, sub_tiles, staged):
    scenes = _scenes(SIZES, 300, bf16)
    b = lib.Batch(scenes, sub_tiles=sub_tiles)
    assert b.plan.pair_path == 0          # odd L in the batch: the general kernel
    b.tuning.dynamic = dynamic
    b.tuning.staged = staged
    b.run()
    lib.nasg_device_status()
    _compare_with_single(lib, scenes)


PAIR_SIZES = [(5001, 8), (777, 16), (12346, 4), (1, 8), (2048, 8), (0, 4), (3, 2), (4093, 4)]


@pytest.mark.parametrize("bf16", [True, False])
@pytest.mark.parametrize("dynamic,sub_tiles,staged", [(1, 1, 0), (0, 3, 0), (1, 1, 1), (0, 2, 1), (1, 8, 1)])
def test_batched_pair_path_equals_single_scene_kernel(lib, bf16, dynamic, sub_tiles, staged):
    """Even L only (the pair-load/store kernel with 32-bit offsets), ragged N, staged and
    direct schedules, scenes whose planes can and cannot be bulk-copied."""
    scenes = _scenes(PAIR_SIZES, 350, bf16)
    b = lib.Batch(scenes, sub_tiles=sub_tiles)
    assert b.plan.pair_path == 1
    b.tuning.dynamic = dynamic
    b.tuning.staged = staged
    b.run()
    lib.nasg_device_status()
    _compare_with_single(lib, scenes)


@pytest.mark.parametrize("bf16", [True, False])
@pytest.mark.parametrize("staged", [0, 1])
def test_batched_many_small_scenes(lib, bf16, staged):
    """256 scenes (the table limit) of 1 .. 300 primitives with L in {2, 4, 8, 16}: the
    scene table in shared memory at its largest, units that end inside a 16-byte unit of
    every buffer, and scenes smaller than one sub-tile."""
    rng = np.random.default_rng(5)
    sizes = [(int(rng.integers(1, 301)), int(rng.choice([2, 4, 8, 16]))) for _ in range(256)]
    scenes = _scenes(sizes, 700, bf16)
    b = lib.Batch(scenes, sub_tiles=2)
    assert b.plan.pair_path == 1
    b.tuning.dynamic = 1
    b.tuning.staged = staged
    b.run()
    lib.nasg_device_status()
    _compare_with_single(lib, scenes[::17])


def test_batched_cos_frames(lib):
    scenes = _scenes([(3000, 8), (1001, 5)], 400, True, "cos")
    b = lib.Batch(scenes, frame_mode="cos")
    b.run()
    _compare_with_single(lib, scenes, "cos")


def test_batched_exact_normalisation(lib):
    scenes = _scenes([(2000, 8), (333, 3), (1024, 16)], 450, True)
    b = lib.Batch(scenes, norm_mode="exact")
    b.tuning.staged = 1
    b.run()
    _compare_with_single(lib, scenes, norm="exact")


def _grads_elementwise(gp, gm, pq, cq, means, cam, g_rgb, L):
    """Every gradient element against the oracle (as the single-scene parity tests):
    |dg| <= 1e-4 |g| + 4 nu + the FP32 floor of the sums of terms of opposite sign."""
    P, n = gp.shape[0], means.shape[0]

    def bwd(p_, c_, m_, cm_):
        r_p, _, r_mu = ong.backward(p_, c_, m_, cm_, g_rgb, L)
        return np.concatenate([r_p.ravel(), r_mu.ravel()])

    ref, nu = sensitivity_floor(bwd, (pq, cq, means, cam), (0, 1, 2, 3))
    groups = np.concatenate([np.repeat(np.arange(P), n * L), np.full(3 * n, P)])
    scale = np.array([np.abs(ref[groups == g]).max() for g in range(P + 1)])
    floor = chain_floor(pq, means, cam, g_rgb, L)
    got = np.concatenate([np.asarray(gp).ravel(), np.asarray(gm).ravel()])
    return grad_report(got, ref, nu, atol=1e-12 * scale[groups] + floor)


def test_batched_oracle_parity(lib):
    import torch
    scenes = _scenes([(2000, 8), (900, 16), (1500, 4)], 500, True)
    b = lib.Batch(scenes)
    assert b.plan.pair_path == 1          # even L only: the pair-load/store kernel
    b.run()
    torch.cuda.synchronize()
    for sc in scenes:
        w, L = sc["w"], sc["n_lobes"]
        pq, cq = inputs.quantize_bf16(w.params), inputs.quantize_bf16(w.c0)
        cam = np.asarray(sc["cam"], np.float32)

        def fwd(p, c, m, cm):
            return ong.forward(p, c, m, cm, L)

        ref, nu = sensitivity_floor(fwd, (pq, cq, w.means, cam), (0, 1, 2, 3))
        rep = colour_report(sc["rgb"].cpu().numpy(), ref, nu, 1e-5)
        assert rep["violations"] == 0, rep
        r_p, _, r_mu = ong.backward(pq, cq, w.means, cam, w.g_rgb, L)
        gp = sc["g_params"].cpu().numpy()
        assert max(rel_l2(gp[p], r_p[p]) for p in range(10)) <= 1e-4
        assert rel_l2(sc["g_means"].cpu().numpy(), r_mu) <= 1e-4
        rep = _grads_elementwise(gp, sc["g_means"].cpu().numpy(), pq, cq, w.means, cam, w.g_rgb, L)
        assert rep["violations"] == 0, rep


def test_batched_full_workload_sampled(lib):
    """The 32-scene batched workload at full size (28M primitives, 2.0e8 BF16 lobes) in
    the launch configuration the benchmark times (autotuned, replayed from a captured
    CUDA graph); the oracle checks a seeded sample of 48 primitives of every scene:
    colours within the usual bound, gradients within relative L2 1e-4 per plane over
    the sample and element by element."""
    import torch
    sizes = inputs.batched_scene_sizes(32, 1004)
    scenes = [inputs.device_point_cloud(n, L, 1004 * 100 + j, "cuda", torch.bfloat16)
              for j, (n, L) in enumerate(sizes)]
    b = lib.Batch(scenes)
    b.autotune(reps=1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    lib.nasg_device_status()
    for j, ((n, L), sc) in enumerate(zip(sizes, scenes)):
        sample = inputs.subsample_indices(n, 48, 31 + j)
        lobes = (sample[:, None] * L + np.arange(L)).reshape(-1)
        ti = torch.from_numpy(sample).cuda()
        tl = torch.from_numpy(lobes).cuda()
        pq = sc["params"][:, tl].float().cpu().numpy()
        cq = sc["c0"][:, ti].float().cpu().numpy()
        ms = sc["means"][ti].cpu().numpy()
        gs = sc["g_rgb"][ti].cpu().numpy()
        cam = np.asarray(sc["cam"], np.float32)

        def fwd(p_, c_, m_, cm_):
            return ong.forward(p_, c_, m_, cm_, L)

        ref, nu = sensitivity_floor(fwd, (pq, cq, ms, cam), (0, 1, 2, 3))
        rep = colour_report(sc["rgb"][ti].cpu().numpy(), ref, nu, 1e-5)
        assert rep["violations"] == 0, (j, rep)
        r_p, r_c0, r_mu = ong.backward(pq, cq, ms, cam, gs, L)
        gp = sc["g_params"][:, tl].cpu().numpy()
        gm = sc["g_means"][ti].cpu().numpy()
        assert max(rel_l2(gp[p], r_p[p]) for p in range(gp.shape[0])) <= 1e-4, j
        np.testing.assert_array_equal(sc["g_c0"][:, ti].cpu().numpy(), r_c0.astype(np.float32))
        assert rel_l2(gm, r_mu) <= 1e-4, j
        rep = _grads_elementwise(gp, gm, pq, cq, ms, cam, gs, L)
        assert rep["violations"] == 0, (j, rep)


def test_batched_cuda_graph_replay_and_autotune(lib):
    import torch
    scenes = _scenes([(20000, 8), (3000, 16), (7000, 4), (50, 8)], 600, True)
    b = lib.Batch(scenes)
    best = b.autotune(reps=2)
    assert best["sub_tiles"] in (1, 2, 4, 8) and best["ms"] > 0
    b.run()
    torch.cuda.synchronize()
    eager = [sc["g_params"].clone() for sc in scenes]
    for sc in scenes:
        sc["g_params"].zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for e, sc in zip(eager, scenes):
        torch.testing.assert_close(sc["g_params"], e, rtol=0, atol=0)


def test_batched_rejects_bad_batches(lib):
    import ctypes
    plan = lib.NasgBatchPlan()
    modes = lib.NasgBatchModes(0, 0, 0, 0)
    arr = (lib.NasgScene * 1)()
    assert lib.lib.nasgabor_batched_prepare(arr, 0, ctypes.byref(modes), 1, ctypes.c_void_p(16), 1 << 20,
                                            ctypes.byref(plan), None) == -2
    assert lib.lib.nasgabor_batched_prepare(arr, 300, ctypes.byref(modes), 1, ctypes.c_void_p(16), 1 << 20,
                                            ctypes.byref(plan), None) == -2
