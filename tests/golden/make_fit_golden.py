"""Writes tests/golden/fit_subsample_20k.json: the FP64 oracle's fit of the
teacher/student workload on a seeded 20,000-primitive subsample.

Workload: 2,000,000 primitives; teacher 4 lobes (FP32 values, seed 1005),
student 16 lobes (seed 1006, stored as BF16 round-to-nearest-even of an FP64
master, as the fused kernel stores it), Adam at base rate 1e-3 times the cosine
schedule factor (Supp. C; oracle.schedule.cosine_factor at iteration step - 1,
starting at iteration 47 of 200), 200 steps, 64 view directions per step shared
by all primitives (inputs.fit_directions(step, 1005)). Primitives are independent, so the subsample's trajectory is that of
the same primitives inside the full run. Recorded: the per-step loss (MSE over
the subsample's primitives, directions and channels, before the step's update),
the final MSE at the held-out step-201 directions, and the same for a pure FP64
fit (no BF16 storage) for information.

Calls only oracle/ and the seeded input generators; run from the repository
root:  python tests/golden/make_fit_golden.py  (about 20 minutes on 8 cores).
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N, LS, LT, STEPS, SAMPLE = 2_000_000, 16, 4, 200, 20_000  # STEPS = inputs.FIT_STEPS
SEED_T, SEED_S, SEED_SAMPLE = 1005, 1006, 7
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fit_subsample_20k.json")


def subsample_workload():
    from paper_2606_09794_gb300 import inputs
    return inputs.fit_subsample(N, LS, LT, SEED_T, SEED_S, SAMPLE, SEED_SAMPLE)


def run_chunk(args):
    tp, tc, sp, sc, bf16 = args
    from paper_2606_09794_gb300 import inputs
    import oracle.adam as oad
    from oracle import schedule
    n = sc.shape[1]
    st = {"student": sp.astype(np.float64), "m": np.zeros(sp.shape), "v": np.zeros(sp.shape),
          "c0": sc.astype(np.float64), "c0_m": np.zeros(sc.shape), "c0_v": np.zeros(sc.shape)}
    sq = []
    for step in range(1, STEPS + 1):
        lr = inputs.FIT_LR * schedule.cosine_factor(step - 1, STEPS, inputs.FIT_SCHEDULE_START)
        new, mse = oad.fit_step(st["student"], st["m"], st["v"], st["c0"], st["c0_m"], st["c0_v"], tp, tc,
                                inputs.fit_directions(step, SEED_T), LS, LT, step, lr=lr, bf16_storage=bf16)
        sq.append(mse * n * 64 * 3)
        st = new
    dirs = inputs.fit_directions(STEPS + 1, SEED_T)
    target = oad.field_colours(tp, tc, dirs, LT)
    p = oad.bf16_round(st["student"]) if bf16 else st["student"]
    c = oad.bf16_round(st["c0"]) if bf16 else st["c0"]
    start_p = oad.bf16_round(sp) if bf16 else sp
    start_c = oad.bf16_round(sc) if bf16 else sc
    final = float(np.sum((oad.field_colours(p, c, dirs, LS) - target) ** 2))
    start = float(np.sum((oad.field_colours(start_p, start_c, dirs, LS) - target) ** 2))
    return np.array(sq), final, start


def main():
    t0 = time.time()
    tp, tc, sp, sc, idx = subsample_workload()
    chunks = 8
    bounds = np.linspace(0, SAMPLE, chunks + 1).astype(int)
    jobs = []
    for bf16 in (True, False):
        for c in range(chunks):
            a, b = bounds[c], bounds[c + 1]
            jobs.append((tp[:, a * LT:b * LT], tc[:, a:b], sp[:, a * LS:b * LS], sc[:, a:b], bf16))
    with mp.get_context("spawn").Pool(min(os.cpu_count() or 1, chunks)) as pool:
        res = pool.map(run_chunk, jobs)
    denom = SAMPLE * 64 * 3
    from paper_2606_09794_gb300 import inputs
    out = {"workload": {"n": N, "student_lobes": LS, "teacher_lobes": LT, "steps": STEPS, "dirs_per_step": 64,
                        "lr": inputs.FIT_LR, "lr_schedule": {"kind": "cosine", "start_iteration": inputs.FIT_SCHEDULE_START,
                                                             "t_max": STEPS, "iteration": "step - 1"},
                        "seed_teacher": SEED_T, "seed_student": SEED_S, "sample": SAMPLE,
                        "seed_sample": SEED_SAMPLE, "final_dirs_step": STEPS + 1},
           "generator": "tests/golden/make_fit_golden.py (FP64 oracle only)"}
    for bf16, key in ((True, "bf16_storage"), (False, "fp64")):
        part = res[:chunks] if bf16 else res[chunks:]
        out[key] = {"loss_per_step": [float(x) for x in sum(r[0] for r in part) / denom],
                    "final_mse": sum(r[1] for r in part) / denom,
                    "start_mse": sum(r[2] for r in part) / denom}
    out["seconds"] = time.time() - t0
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(OUT, out["bf16_storage"]["final_mse"], out["fp64"]["final_mse"], out["seconds"])


if __name__ == "__main__":
    main()
