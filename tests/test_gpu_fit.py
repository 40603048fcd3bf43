"""GPU parity of the teacher-student fitting step against the FP64 oracle
(oracle/adam.py fit_step: per-primitive mean squared colour error over the
shared directions, gradient summed over them, one Adam step, BF16 storage).
The 200-step runs take the workload's learning-rate schedule: base rate 1e-3
times the cosine factor (Supp. C) from iteration 47 on, formed by the library's
nasg_cosine_lr_factor on the GPU side and by oracle.schedule on the oracle side."""
import numpy as np
import pytest

from oracle import adam as oad
from oracle import schedule as osch
from paper_2606_09794_gb300 import inputs
from tests._parity import adam_consistency, rel_l2

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _lr_gpu(lib, step):
    return inputs.FIT_LR * lib.nasg_cosine_lr_factor(step - 1, inputs.FIT_STEPS, inputs.FIT_SCHEDULE_START)


def _lr_oracle(step):
    return inputs.FIT_LR * osch.cosine_factor(step - 1, inputs.FIT_STEPS, inputs.FIT_SCHEDULE_START)


def _setup(lib, n, ls, lt, seed, warm):
    t = inputs.point_cloud_workload(n, lt, seed)
    s = inputs.point_cloud_workload(n, ls, seed + 1)
    rng = np.random.default_rng(seed)
    m = (0.01 * rng.standard_normal(s.params.shape)).astype(np.float32) if warm else np.zeros_like(s.params)
    v = (1e-4 * (1 + rng.random(s.params.shape))).astype(np.float32) if warm else np.zeros_like(s.params)
    cm = (0.01 * rng.standard_normal(s.c0.shape)).astype(np.float32) if warm else np.zeros_like(s.c0)
    cv = (1e-4 * (1 + rng.random(s.c0.shape))).astype(np.float32) if warm else np.zeros_like(s.c0)
    st = lib.TrainState(_dev(s.params), _dev(s.c0), _dev(m), _dev(v), _dev(cm), _dev(cv))
    return t, s, st, (m, v, cm, cv)


@pytest.mark.parametrize("ls,lt,ndirs,norm", [(16, 4, 64, "approx"), (8, 4, 13, "approx"), (4, 2, 7, "approx"),
                                             (8, 4, 9, "exact")])
def test_fit_steps_match_oracle(lib, ls, lt, ndirs, norm):
    n = 96
    t, s, st, (m, v, cm, cv) = _setup(lib, n, ls, lt, 41 + ls, warm=True)
    tp, tc = _dev(t.params), _dev(t.c0)
    state = {"student": s.params.astype(np.float64), "m": m.astype(np.float64), "v": v.astype(np.float64),
             "c0": s.c0.astype(np.float64), "c0_m": cm.astype(np.float64), "c0_v": cv.astype(np.float64)}
    for step in (1, 2, 150):             # the last at a scheduled rate (factor ~0.3)
        dirs = inputs.fit_directions(step, 7, ndirs)
        lr = _lr_gpu(lib, step)
        assert lr == pytest.approx(_lr_oracle(step), rel=1e-15)
        loss = lib.nasgabor_fit_step(st, tp, tc, lt, _dev(dirs), ls, step, lr=lr, norm_mode=norm)
        new, mse = oad.fit_step(state["student"], state["m"], state["v"], state["c0"], state["c0_m"], state["c0_v"],
                                t.params, t.c0, dirs, ls, lt, step, lr=_lr_oracle(step), norm_mode=norm)
        assert abs(float(loss.item()) - mse) <= 1e-4 * mse + 1e-9, (float(loss.item()), mse)
        # moments (the gradient summed over the directions) against the oracle; every new
        # value against the Adam update from the GPU's own moments to one FP32 ulp; the
        # update against the oracle's within 2e-3, the moments' 1e-4 plus the FP32
        # rounding of the new value (up to 2.4e-4 of a 1e-3 step at |theta| ~ 7) and the
        # summed gradient's cancellation between directions
        got = st.master.cpu().numpy().astype(np.float64)
        m_gpu, v_gpu = st.m.cpu().numpy(), st.v.cpu().numpy()
        for p in range(10):
            rep = adam_consistency(got[p], state["student"][p], m_gpu[p], v_gpu[p], step, lr=np.float32(lr))
            assert rep["violations"] == 0, (step, p, rep)
            d_gpu = got[p] - state["student"][p]
            d_ref = new["student"][p] - state["student"][p]
            assert rel_l2(d_gpu, d_ref) < 2e-3, (step, p, rel_l2(d_gpu, d_ref))
        assert rel_l2(m_gpu, new["m"]) < 1e-4 and rel_l2(v_gpu, new["v"]) < 1e-4
        # continue both from the GPU's state so that the comparison stays one step deep
        state = {"student": got, "m": st.m.cpu().numpy().astype(np.float64), "v": st.v.cpu().numpy().astype(np.float64),
                 "c0": st.c0_master.cpu().numpy().astype(np.float64),
                 "c0_m": st.c0_m.cpu().numpy().astype(np.float64), "c0_v": st.c0_v.cpu().numpy().astype(np.float64)}
    import torch
    torch.testing.assert_close(st.params_bf16, st.master.to(torch.bfloat16), rtol=0, atol=0)


def test_fit_run_matches_oracle_fit_on_a_sample(lib):
    """200 steps of 64 directions on 4096 primitives (L_s = 16 BF16, L_t = 4 FP32) at the
    scheduled rates; the oracle runs the same fit from the same start on a seeded sample
    of 64 primitives (primitives are independent); final per-sample MSE within 1 %."""
    n, ls, lt, steps = 4096, 16, 4, 200
    t, s, st, _ = _setup(lib, n, ls, lt, 1005, warm=False)
    tp, tc = _dev(t.params), _dev(t.c0)
    for step in range(1, steps + 1):
        lib.nasgabor_fit_step(st, tp, tc, lt, _dev(inputs.fit_directions(step, 1005)), ls, step,
                              lr=_lr_gpu(lib, step))
    sample = inputs.subsample_indices(n, 64, 3)
    lobes_s = (sample[:, None] * ls + np.arange(ls)).reshape(-1)
    lobes_t = (sample[:, None] * lt + np.arange(lt)).reshape(-1)
    tps, tcs = t.params[:, lobes_t], t.c0[:, sample]
    P = s.params.shape[0]
    stt = {"student": s.params[:, lobes_s].astype(np.float64), "m": np.zeros((P, len(lobes_s))),
           "v": np.zeros((P, len(lobes_s))), "c0": s.c0[:, sample].astype(np.float64),
           "c0_m": np.zeros((3, len(sample))), "c0_v": np.zeros((3, len(sample)))}
    for step in range(1, steps + 1):
        new, _ = oad.fit_step(stt["student"], stt["m"], stt["v"], stt["c0"], stt["c0_m"], stt["c0_v"], tps, tcs,
                              inputs.fit_directions(step, 1005), ls, lt, step, lr=_lr_oracle(step))
        stt = new
    # final MSE of the sample, evaluated by the oracle for both final states
    dirs = inputs.fit_directions(steps + 1, 1005)
    target = oad.field_colours(tps, tcs, dirs, lt)
    gpu_p = st.master.cpu().numpy()[:, lobes_s].astype(np.float64)
    gpu_c = st.c0_master.cpu().numpy()[:, sample].astype(np.float64)
    mse_gpu = np.mean((oad.field_colours(oad.bf16_round(gpu_p), oad.bf16_round(gpu_c), dirs, ls) - target) ** 2)
    mse_ref = np.mean((oad.field_colours(oad.bf16_round(stt["student"]), oad.bf16_round(stt["c0"]), dirs, ls)
                       - target) ** 2)
    start = np.mean((oad.field_colours(oad.bf16_round(s.params[:, lobes_s]), oad.bf16_round(s.c0[:, sample]), dirs, ls)
                     - target) ** 2)
    assert mse_ref < 0.9 * start  # the fit makes progress
    assert abs(mse_gpu - mse_ref) <= 0.01 * mse_ref, (mse_gpu, mse_ref, start)


def test_fit_subsample_matches_stored_oracle_fit(lib):
    """The full fitting workload's 20,000-primitive subsample (2M primitives, 16-lobe
    BF16 student, 4-lobe teacher, 64 directions, 200 Adam steps at the scheduled rates): the
    GPU's per-step loss and its loss at the held-out step-201 directions against the
    FP64 oracle's fit stored by tests/golden/make_fit_golden.py (1 %)."""
    import importlib.util
    import json
    import os

    import torch
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_fit_golden", os.path.join(here, "make_fit_golden.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    with open(os.path.join(here, "fit_subsample_20k.json")) as f:
        gold = json.load(f)
    tp, tc, sp, sc, _ = gen.subsample_workload()
    st = lib.TrainState(_dev(sp), _dev(sc))
    tpd, tcd = _dev(tp), _dev(tc)
    steps = gold["workload"]["steps"]
    losses = torch.empty(steps + 1, device="cuda")
    assert gold["workload"]["lr_schedule"]["start_iteration"] == inputs.FIT_SCHEDULE_START
    for step in range(1, steps + 2):
        lib.nasgabor_fit_step(st, tpd, tcd, gen.LT, _dev(inputs.fit_directions(step, gen.SEED_T)), gen.LS, step,
                              lr=_lr_gpu(lib, step), loss=losses[step - 1:step])
    got = losses.cpu().numpy().astype(np.float64)
    ref = np.asarray(gold["bf16_storage"]["loss_per_step"])
    rel = np.abs(got[:steps] - ref) / ref
    assert rel.max() <= 0.01, (rel.max(), int(rel.argmax()))
    final = gold["bf16_storage"]["final_mse"]
    assert abs(got[steps] - final) <= 0.01 * final, (got[steps], final)
    assert got[steps] < 0.9 * gold["bf16_storage"]["start_mse"]
