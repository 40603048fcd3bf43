"""GPU parity of the frustum compaction and the fused forward+backward+Adam step
against the FP64 oracle (oracle/frustum.py, oracle/adam.py).

Visibility is an integer decision: the index lists must agree exactly except for
centres within a float32 rounding margin of a frustum face, where either answer
is valid. The step: the Adam moments within relative L2 1e-4 per plane of the
oracle (which evaluates at the dequantised BF16 values); every new parameter value
equal, to one FP32 ulp, to the Adam update formed from the GPU's own new moments
(adam_consistency); the update itself against the oracle's within relative L2
1e-3 per plane, which is the moments' 1e-4 plus the FP32 rounding of the new value
(up to ulp/2 = 2.4e-7 at |theta| ~ 7, 2.4e-4 of a 1e-3 step); the BF16 copy
bit-equal to RNE(FP32 master); untouched primitives bit-identical.
"""
import numpy as np
import pytest

from oracle import adam as oad
from oracle import frustum as ofr
from oracle import nasgabor as ong
from paper_2606_09794_gb300 import inputs
from tests._parity import adam_consistency, colour_report, rel_l2, sensitivity_floor

pytestmark = pytest.mark.gpu

MARGIN = 1e-5


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _compact(lib, means_np, cam):
    import torch
    idx, nv = lib.nasg_frustum_compact(_dev(means_np), cam.rot, cam.center, cam.tan_half_fov)
    torch.cuda.synchronize()
    k = int(nv.item())
    return idx[:k].cpu().numpy(), idx, nv


def _check_visibility(got, means, cam):
    ref = ofr.visible(means, cam.rot, cam.center, cam.tan_half_fov)
    margin = ofr.boundary_margin(means, cam.rot, cam.center, cam.tan_half_fov)
    assert np.all(np.diff(got) > 0)  # ascending, unique
    mask = np.zeros(len(means), bool)
    mask[got] = True
    bad = (mask != ref) & (margin > MARGIN)
    assert not bad.any(), np.flatnonzero(bad)[:10]


@pytest.mark.parametrize("n", [1, 4095, 4096, 4097, 100_003])
def test_frustum_compaction(lib, n):
    sc = inputs.shell_scene(n, 1, 77, fov_sample=min(n, 50_000))
    for cam in sc.cameras[:3]:
        got, _, _ = _compact(lib, sc.means, cam)
        _check_visibility(got, sc.means, cam)


def test_frustum_compaction_edge_cases(lib):
    import torch
    sc = inputs.shell_scene(5000, 1, 78, fov_sample=5000)
    cam = sc.cameras[0]
    wide = inputs.RingCamera(cam.center, cam.rot, 1e6)
    got, _, _ = _compact(lib, sc.means, wide)
    ref = ofr.visible(sc.means, wide.rot, wide.center, wide.tan_half_fov)
    np.testing.assert_array_equal(got, np.flatnonzero(ref))
    behind = inputs.RingCamera(cam.center, -cam.rot, cam.tan_half_fov)  # looking away: nothing in front
    got, _, _ = _compact(lib, sc.means, behind)
    assert got.size == 0
    idx, nv = lib.nasg_frustum_compact(torch.zeros((0, 3), device="cuda"), cam.rot, cam.center, 0.5)
    assert int(nv.item()) == 0


def _state(lib, w_params, c0, seed, warm):
    """Optimiser state with non-zero moments (so the update is smooth in g)."""
    import torch
    rng = np.random.default_rng(seed)
    m = (0.01 * rng.standard_normal(w_params.shape)).astype(np.float32) if warm else np.zeros_like(w_params)
    v = (1e-4 * (1 + rng.random(w_params.shape))).astype(np.float32) if warm else np.zeros_like(w_params)
    cm = (0.01 * rng.standard_normal(c0.shape)).astype(np.float32) if warm else np.zeros_like(c0)
    cv = (1e-4 * (1 + rng.random(c0.shape))).astype(np.float32) if warm else np.zeros_like(c0)
    st = lib.TrainState(_dev(w_params), _dev(c0), _dev(m), _dev(v), _dev(cm), _dev(cv))
    return st, (w_params.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                c0.astype(np.float64), cm.astype(np.float64), cv.astype(np.float64))


@pytest.mark.parametrize("L,frame,n,norm,loss", [(8, "quat", 3000, "approx", "given"),
                                                 (5, "quat", 1001, "approx", "given"),
                                                 (4, "cos", 2000, "approx", "given"),
                                                 (6, "quat", 1500, "exact", "given"),
                                                 (8, "quat", 3000, "approx", "mse"),
                                                 (5, "quat", 1001, "approx", "mse"),
                                                 (4, "cos", 2000, "exact", "mse")])
def test_fused_step_matches_oracle(lib, L, frame, n, norm, loss):
    """One step from a warm state. loss "mse": the kernel forms dLoss/dc = 2 (c - t) /
    (3 n_listed) from each listed primitive's colour and a target colour t ~ U[0, 2]^3."""
    import torch
    sc = inputs.shell_scene(n, L, 90 + L, frame_mode=frame, fov_sample=n)
    cam = sc.cameras[1]
    g = inputs.ring_upstream(n, 1, 90 + L)
    if loss == "mse":
        g = np.random.default_rng(91 + L).uniform(0.0, 2.0, (n, 3)).astype(np.float32)
    # MSE gradients are ~1/n_listed: from a cold state m = (1 - b1) g tests them directly
    st, (p0, m0, v0, c00, cm0, cv0) = _state(lib, sc.params, sc.c0, 5, warm=(loss == "given"))
    idx_full, nv = lib.nasg_frustum_compact(_dev(sc.means), cam.rot, cam.center, cam.tan_half_fov)
    rgb = torch.full((n, 3), -3.0, device="cuda")
    t = 7
    lib.nasgabor_fused_step(st, _dev(sc.means), cam.center, _dev(g), L, t, lr=1e-3, idx=idx_full,
                            n_idx_device=nv, frame_mode=frame, norm_mode=norm, rgb=rgb, loss=loss)
    lib.nasg_device_status()
    vis = idx_full[:int(nv.item())].cpu().numpy()
    _check_visibility(vis, sc.means, cam)
    out = oad.fused_step(p0, m0, v0, c00, cm0, cv0, sc.means, cam.center, g, vis, L, t, lr=1e-3,
                         frame_mode=frame, norm_mode=norm, loss=loss)
    master = st.master.cpu().numpy().astype(np.float64)
    P = master.shape[0]
    lobes = (vis[:, None] * L + np.arange(L)).reshape(-1)
    hidden = np.setdiff1d(np.arange(n * L), lobes)
    # untouched primitives: bit-identical state
    np.testing.assert_array_equal(st.master.cpu().numpy()[:, hidden], sc.params[:, hidden])
    np.testing.assert_array_equal(st.m.cpu().numpy()[:, hidden], m0[:, hidden].astype(np.float32))
    # updated primitives against the oracle
    m_gpu, v_gpu = st.m.cpu().numpy(), st.v.cpu().numpy()
    for p in range(P):
        assert rel_l2(m_gpu[p, lobes], out["m"][p, lobes]) < 1e-4, p
        assert rel_l2(v_gpu[p, lobes], out["v"][p, lobes]) < 1e-4, p
        rep = adam_consistency(master[p, lobes], p0[p, lobes], m_gpu[p, lobes], v_gpu[p, lobes], t)
        assert rep["violations"] == 0, (p, rep)
        assert rel_l2(master[p, lobes] - p0[p, lobes], out["master"][p, lobes] - p0[p, lobes]) < 1e-3, p
    c0n, c0m, c0v = (x.cpu().numpy()[:, vis] for x in (st.c0_master, st.c0_m, st.c0_v))
    assert rel_l2(c0m, out["c0_m"][:, vis]) < 1e-4 and rel_l2(c0v, out["c0_v"][:, vis]) < 1e-4
    rep = adam_consistency(c0n, c00[:, vis], c0m, c0v, t)
    assert rep["violations"] == 0, rep
    assert rel_l2(c0n - c00[:, vis], out["c0"][:, vis] - c00[:, vis]) < 1e-3
    # BF16 copies are the RNE of the updated FP32 master
    torch.testing.assert_close(st.params_bf16, st.master.to(torch.bfloat16), rtol=0, atol=0)
    torch.testing.assert_close(st.c0_bf16, st.c0_master.to(torch.bfloat16), rtol=0, atol=0)
    # colours of the listed primitives at the BF16 values
    pq = inputs.quantize_bf16(sc.params[:, lobes].astype(np.float32))
    cq = inputs.quantize_bf16(sc.c0[:, vis])

    def fwd(p_, c_, m_, cam_):
        return ong.forward(p_, c_, m_, cam_, L, frame, norm)

    ref, nu = sensitivity_floor(fwd, (pq, cq, sc.means[vis], cam.center), (0, 1, 2, 3))
    rep = colour_report(rgb.cpu().numpy()[vis], ref, nu, 1e-5)
    assert rep["violations"] == 0, rep
    assert (rgb.cpu().numpy()[np.setdiff1d(np.arange(n), vis)] == -3.0).all()


@pytest.mark.parametrize("n,order,fov_sample", [(400_000, "random", 100_000), (6_000_000, "morton", 200_000)])
def test_ring_of_cameras_sampled(lib, n, order, fov_sample):
    """The scene-scale workload, at reduced N in random storage order and at the full
    6e6 in the Morton order the benchmark times: 8 cameras back to back, one step each
    (global step counter, cold optimiser state), then a seeded sample of primitives
    replayed by the oracle (primitives are independent; samples near a frustum face are
    excluded)."""
    import torch
    L = 8
    sc = inputs.shell_scene(n, L, 1003, fov_sample=fov_sample, order=order)
    st = lib.TrainState(_dev(sc.params), _dev(sc.c0))
    means = _dev(sc.means)
    ws = torch.empty(lib.nasg_frustum_workspace_bytes(n), device="cuda", dtype=torch.uint8)
    idx = torch.empty(n, device="cuda", dtype=torch.int32)
    nv = torch.empty(1, device="cuda", dtype=torch.int32)
    gs = [inputs.ring_upstream(n, j, 1003) for j in range(len(sc.cameras))]
    for j, cam in enumerate(sc.cameras):
        lib.nasg_frustum_compact(means, cam.rot, cam.center, cam.tan_half_fov, idx=idx, n_visible=nv, workspace=ws)
        lib.nasgabor_fused_step(st, means, cam.center, _dev(gs[j]), L, j + 1, idx=idx, n_idx_device=nv)
    lib.nasg_device_status()
    sample = inputs.subsample_indices(n, 400, 9)
    margins = np.min([ofr.boundary_margin(sc.means[sample], c.rot, c.center, c.tan_half_fov)
                      for c in sc.cameras], axis=0)
    sample = sample[margins > MARGIN]
    lobes = (sample[:, None] * L + np.arange(L)).reshape(-1)
    P = sc.params.shape[0]
    init_p = sc.params[:, lobes].astype(np.float64)
    mast = init_p.copy()
    m = np.zeros_like(mast)
    v = np.zeros_like(mast)
    c0 = sc.c0[:, sample].astype(np.float64)
    cm = np.zeros_like(c0)
    cv = np.zeros_like(c0)
    ms = sc.means[sample]
    for j, cam in enumerate(sc.cameras):
        vis = np.flatnonzero(ofr.visible(ms, cam.rot, cam.center, cam.tan_half_fov))
        out = oad.fused_step(mast, m, v, c0, cm, cv, ms, cam.center, gs[j][sample], vis, L, j + 1)
        mast, m, v, c0, cm, cv = out["master"], out["m"], out["v"], out["c0"], out["c0_m"], out["c0_v"]
    # after 8 steps the two trajectories differ by the FP32 rounding of each new value
    # (<= 2.4e-7 per step at |theta| ~ 7 against steps of ~1e-3), and a master that ends
    # within that distance of a BF16 rounding boundary is evaluated one BF16 ulp apart on
    # the next step (about 5e-5 of the 2.6e5 lobe-plane-steps here): the total update of
    # each plane within relative L2 2e-3 (the single-step test checks each step tightly)
    got = st.master[:, torch.from_numpy(lobes).cuda()].cpu().numpy().astype(np.float64)
    assert len(sample) > 200
    for p in range(P):
        assert rel_l2(got[p] - init_p[p], mast[p] - init_p[p]) < 2e-3, p
    torch.testing.assert_close(st.params_bf16, st.master.to(torch.bfloat16), rtol=0, atol=0)


@pytest.mark.parametrize("n,L,offset", [(1000, 8, 0), (777, 3, 0), (64, 8, 1), (1, 1, 0)])
def test_train_state_bf16_copies_are_rne(lib, n, L, offset):
    """nasg_train_state_refresh_bf16 writes RNE_bf16 of the masters, bit for bit as torch's
    rounding cast, incl. exact halfway cases (both parities), +-0, subnormals, infinities,
    and on the element path (an offset view breaks the 16-byte alignment of the vector path)."""
    import torch
    rng = np.random.default_rng(n + L)
    bits = rng.integers(0, 2 ** 32, size=10 * n * L + 3 * n, dtype=np.uint64).astype(np.uint32)
    bits[0::7] = (bits[0::7] & 0xFFFF0000) | 0x8000            # exact ties
    vals = bits.view(np.float32).copy()
    vals[~np.isfinite(vals)] = 1.5
    vals[:8] = np.array([0.0, -0.0, 1e-40, -1e-42, np.inf, -np.inf, 3.4e38, 1.0 + 2 ** -8], np.float32)
    big = torch.from_numpy(np.concatenate([np.zeros(offset, np.float32), vals])).cuda()
    flat = big[offset:]
    master = flat[:10 * n * L].view(10, n * L)
    c0 = flat[10 * n * L:].view(3, n)
    st = lib.TrainState(master, c0)
    lib.nasg_device_status()
    torch.testing.assert_close(st.params_bf16.view(torch.int16), master.to(torch.bfloat16).view(torch.int16),
                               rtol=0, atol=0)
    torch.testing.assert_close(st.c0_bf16.view(torch.int16), c0.to(torch.bfloat16).view(torch.int16), rtol=0, atol=0)
