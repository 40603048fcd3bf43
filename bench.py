#!/usr/bin/env python3
"""Throughput of the NASGabor appearance path on GB300: primitives*lobes/s.

Headline step: one fused forward+backward pass (given upstream dLoss/dRGB) of
the NASGabor appearance model over N = 1,000,000 primitives with L = 8 lobes,
parameters stored in BF16 (FP32 math), QUAT frames, approximate normalisation,
on synthetic primitives (seeded; unit-cube positions, one camera at (0,0,3)).
One step = one launch of the fused kernel. value = N*L*steps / time.

Side measurements in the same JSON line ("paths"): the plain FP32 path
(separate forward and backward kernels), the FP32 fused kernel and the SH
degree-3 comparison kernels at the same N and view directions, each with its
kernels' HBM roofline fraction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank times its own shard of the same size (weak scaling,
no collective on the data path); the timing is max-reduced over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_PRIMS = 1_000_000
N_LOBES = 8
SEED = 1002
E2E_CHUNK = 131072
METRIC = "primitives*lobes/s fwd+bwd (fused BF16-parameter NASGabor)"
UNIT = "primitive-lobes/s"
FALLBACK_HBM_GBS = 6800.0

# Algorithmic bytes per primitive (QUAT, P = 10 raw scalars per lobe):
#   fused BF16 fwd+bwd: per lobe 20 B params read + 40 B f32 gradients written;
#     per primitive mu 12 + c0 6 + g_rgb 12 read, rgb 12 + g_c0 12 + g_mu 12 written.
#   fused FP32 fwd+bwd: per lobe 40 + 40; per primitive 12 + 12 + 12 + 12 + 12 + 12.
#   plain FP32 fwd: per lobe 40; per primitive mu 12 + c0 12 + rgb 12.
#   plain FP32 bwd: per lobe 40 + 40; per primitive mu 12 + g_rgb 12 + g_c0 12 + g_mu 12.
#   SH-3 fwd: 48 coefficients * 4 B + mu 12 + rgb 12; SH-3 bwd: coefficients read
#     (for dLoss/dmu) 192 + g_coeffs 192 + mu 12 + g_rgb 12 + g_mu 12.


def bytes_fused_bf16(L):
    return 60 * L + 66


def bytes_fused_f32(L):
    return 80 * L + 72


def bytes_fwd_f32(L):
    return 40 * L + 36


def bytes_bwd_f32(L):
    return 80 * L + 48


BYTES_SH3_FWD = 216
BYTES_SH3_BWD = 420


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    """Hash of every source the headline kernel is compiled from (csrc/nasg_*.cuh, nasg_*.h, nasg_eval*.cu)."""
    csrc = os.path.join(ROOT, "paper_2606_09794_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(csrc)):
        if (f.startswith("nasg_") and (f.endswith(".cuh") or f.endswith(".h"))) or \
                (f.startswith("nasg_eval") and f.endswith(".cu")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the headline kernel from the committed ncu summary,
    or None when the kernel source has changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "nasgabor_fused_bf16_fwd_bwd_1m_l8.md")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if line.startswith("- ") and ":" in line:
                    k, v = line[2:].split(":", 1)
                    kv[k.strip()] = v.strip().strip("`")
        if kv.get("source_sha256_16") != kernel_source_hash():
            return None
        return int(float(kv["dram_bytes_per_launch"]))
    except Exception:
        return None


# ---------------------------------------------------------------------------
# distributed helpers (host logic; tested with gloo on CPU)
# ---------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_seed(base_seed, rank):
    """Every rank gets its own shard of the same size and distribution."""
    return base_seed + 7919 * rank


def reduce_max(value, world, device=None):
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.samples = []
        self.proc = None
        self.thread = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                self.samples.append((time.time(), float(parts[0]), float(parts[1]), parts[3:8]))
            except ValueError:
                continue

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        inside = [s for s in self.samples if t0 <= s[0] <= t1]
        window = "timed"
        if len(inside) < 3:
            inside = [s for s in self.samples if s[0] <= t1]
            window = "warmup+timed"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for s in inside:
            for nm, v in zip(names, s[3][1:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(s[1] for s in inside), "sm_max_mhz": max(s[2] for s in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


def gpu_id_for_smi(local_rank):
    """nvidia-smi -i argument for the device this rank runs on (its UUID when torch knows it)."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local_rank).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[local_rank] if vis else str(local_rank)


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on a bounded sample
# ---------------------------------------------------------------------------

def cpu_oracle_rate(target_s=12.0, max_n=100_000):
    """Oracle forward+backward (BF16-dequantised parameters) on a seeded sample of
    the headline workload, sized for about target_s of single-thread CPU work."""
    try:
        from threadpoolctl import threadpool_limits
    except Exception:  # pragma: no cover - not in every image
        threadpool_limits = None
    import contextlib

    import numpy as np

    from oracle import nasgabor as ong
    from paper_2606_09794_gb300 import inputs

    ctx = threadpool_limits(limits=1) if threadpool_limits else contextlib.nullcontext()
    L = N_LOBES

    def run(n):
        w = inputs.point_cloud_workload(n, L, SEED)
        p = inputs.quantize_bf16(w.params)
        c = inputs.quantize_bf16(w.c0)
        t0 = time.perf_counter()
        ong.forward(p, c, w.means, w.cam, L)
        ong.backward(p, c, w.means, w.cam, w.g_rgb, L)
        return time.perf_counter() - t0

    with ctx:
        probe_n = 2000
        dt = run(probe_n)
        n = int(min(max_n, max(probe_n, probe_n * target_s / max(dt, 1e-6))))
        reps, total = 0, 0.0
        while total < target_s or reps == 0:
            total += run(n)
            reps += 1
    return {"value": n * L * reps / total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} primitives x {L} lobes of the N=1e6 workload (seed {SEED}) x {reps} passes, "
                      f"forward+backward in float64 numpy, one thread, {total:.1f} s"}


def _oracle_worker(args):
    """One host process of the all-cores oracle timing: forward+backward passes of the
    FP64 oracle (one thread) on its own seeded slice for about target_s seconds."""
    n, seed, target_s = args
    try:
        from threadpoolctl import threadpool_limits
        ctx = threadpool_limits(limits=1)
    except Exception:  # pragma: no cover
        import contextlib
        ctx = contextlib.nullcontext()
    from oracle import nasgabor as ong
    from paper_2606_09794_gb300 import inputs
    L = N_LOBES
    w = inputs.point_cloud_workload(n, L, seed)
    p = inputs.quantize_bf16(w.params)
    c = inputs.quantize_bf16(w.c0)
    reps, t0 = 0, time.perf_counter()
    with ctx:
        while time.perf_counter() - t0 < target_s or reps == 0:
            ong.forward(p, c, w.means, w.cam, L)
            ong.backward(p, c, w.means, w.cam, w.g_rgb, L)
            reps += 1
    return n * L * reps, time.perf_counter() - t0


def cpu_oracle_rate_all_cores(target_s=8.0, n_per_proc=20_000):
    """The same oracle pass on every host core at once (one process per core,
    started with spawn), for context next to the one-thread baseline."""
    import multiprocessing as mp
    procs = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(n_per_proc, SEED + 1 + k, target_s) for k in range(procs)])
    lobes = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": lobes / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes x {n_per_proc} primitives x {N_LOBES} lobes (seeded slices of the "
                      f"N=1e6 workload), forward+backward in float64 numpy, one thread each, {wall:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    vals = []
    per_step = float(os.environ.get("BENCH_ORACLE_TARGET_S", max(2.0, 20.0 / max(args.steps, 1))))
    for _ in range(args.warmup):
        cpu_oracle_rate(target_s=min(2.0, per_step))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_oracle_rate(target_s=per_step))
    wall = time.perf_counter() - t0
    value = statistics.median(v["value"] for v in vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"NASGabor fwd+bwd, N={N_PRIMS}, L={N_LOBES}, QUAT, BF16-stored params "
                               "(sampled per step)", "global_batch": N_PRIMS, "lobes": N_LOBES},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1,
                         "sample": vals[-1]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU measurement
# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paths", action="store_true")
    ap.add_argument("--case", choices=["paths", "scene_step", "batched", "batched_one", "fit", "frame"], default=None,
                    help="run only this secondary measurement (at --case-n primitives) and print its JSON")
    ap.add_argument("--case-n", type=int, default=None)
    ap.add_argument("--case-steps", type=int, default=None)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)
    if args.warmup < 3:
        args.warmup = 3

    import numpy as np
    import torch

    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_2606_09794_gb300 import binding as nb
    from paper_2606_09794_gb300 import inputs

    N, L = N_PRIMS, N_LOBES
    w = inputs.point_cloud_workload(N, L, shard_seed(SEED, rank))
    params = torch.from_numpy(w.params).to(dev).to(torch.bfloat16)
    c0 = torch.from_numpy(w.c0).to(dev).to(torch.bfloat16)
    means = torch.from_numpy(w.means).to(dev)
    g_rgb = torch.from_numpy(w.g_rgb).to(dev)
    cam = tuple(float(x) for x in w.cam)
    out = (torch.empty((N, 3), device=dev), torch.empty(params.shape, device=dev, dtype=torch.float32),
           torch.empty((3, N), device=dev), torch.empty((N, 3), device=dev))
    stream = torch.cuda.current_stream(dev)

    def step():
        nb.nasgabor_fused_fwd_bwd(params, c0, means, cam, g_rgb, L, out=out, stream=stream)

    peak, peak_kind = load_peaks()
    sampler = ClockSampler(gpu_id_for_smi(local_rank)) if rank == 0 else None
    time.sleep(0.3)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    t_wall0 = time.time()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize(dev)
    t_wall1 = time.time()
    barrier(world, dev)
    ms_local = ev0.elapsed_time(ev1)
    ms = reduce_max(ms_local, world, dev)
    clocks = sampler.summary(t_wall0, t_wall1) if sampler else None
    if sampler:
        sampler.stop()

    units = N * L * args.steps * world
    value = units / (ms * 1e-3)
    ms_per_step = ms / args.steps
    alg_bytes = N * bytes_fused_bf16(L)
    achieved = alg_bytes / (ms_local / args.steps * 1e-3) / 1e9
    traffic = profiled_traffic()

    # ---- end to end through the public API with host buffers -------------------
    # the C-ABI call on HOST (pinned) arrays: the library streams the primitives in
    # chunks through the device, copies in both directions overlapping the kernel
    pin = dict(params=params.cpu().pin_memory(), c0=c0.cpu().pin_memory(), means=means.cpu().pin_memory(),
               g_rgb=g_rgb.cpu().pin_memory())
    host_out = tuple(torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in out)
    h2d = sum(t.numel() * t.element_size() for t in pin.values())
    d2h = sum(t.numel() * t.element_size() for t in host_out)
    host_fused = nb.HostFused(N, L, params.dtype, chunk=E2E_CHUNK, device=dev)

    def e2e_step():
        host_fused(pin["params"], pin["c0"], pin["means"], cam, pin["g_rgb"], host_out, stream=stream)

    e2e_steps = max(5, min(50, args.steps))
    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    e1.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1), world, dev)
    e2e_value = N * L * e2e_steps * world / (e2e_ms * 1e-3)

    paths = None
    if rank == 0 and world == 1 and not args.no_paths:
        paths = measure_paths(nb, inputs, w, params, dev, stream, peak)
        del w
        paths["scene_step"] = measure_scene_step(nb, inputs, dev, stream, peak)
        paths["batched"] = measure_batched(nb, inputs, dev, stream, peak)
        paths["fit"] = measure_fit(nb, inputs, dev, stream)
        paths["frame"] = measure_frame(nb, inputs, dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate()
        if paths is not None:
            paths["cpu_oracle_all_cores"] = cpu_oracle_rate_all_cores()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"NASGabor fused fwd+bwd, N={N} primitives per GPU, L={L} lobes, QUAT "
                                   "frames, BF16-stored params, FP32 math, approx. normalisation, "
                                   "upstream dL/dRGB ~ N(0,1)",
                       "global_batch": N * world, "lobes": L, "param_storage": "bf16",
                       "parallelism": f"replicas x{world} (independent shards)",
                       "l2": "no flush: inputs 190 MB + outputs 356 MB per step exceed the 129 MB L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "eval_tma_kernel<QUAT, bf16, fwd+bwd, default flags>",
                         "algorithmic_bytes_per_launch": alg_bytes},
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "api": "nasgabor_fused_fwd_bwd_host (host arrays, chunks of "
                                                f"{E2E_CHUNK} primitives)"},
            "gpu_launches": args.steps,
            "cpu_baseline": cpu,
            "paths": paths,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_case(args):
    """One secondary measurement on its own (used for profiling captures of a smaller case)."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2606_09794_gb300 import binding as nb
    from paper_2606_09794_gb300 import inputs
    stream = torch.cuda.current_stream(dev)
    peak, _ = load_peaks()
    kw = {}
    if args.case_n:
        kw["n"] = args.case_n
    if args.case == "paths":
        n = args.case_n or N_PRIMS
        w = inputs.point_cloud_workload(n, N_LOBES, SEED)
        params = torch.from_numpy(w.params).to(dev).to(torch.bfloat16)
        res = measure_paths(nb, inputs, w, params, dev, stream, peak, reps=args.case_steps or 200)
    elif args.case == "scene_step":
        res = measure_scene_step(nb, inputs, dev, stream, peak, **kw)
    elif args.case == "frame":
        res = measure_frame(nb, inputs, dev, stream, **kw)
    elif args.case == "batched":
        res = measure_batched(nb, inputs, dev, stream, peak, **({"n_scenes": args.case_n} if args.case_n else {}))
    elif args.case == "batched_one":
        res = measure_batched_one(nb, inputs, dev, stream, peak, **({"n_lobes": args.case_n} if args.case_n else {}),
                                  **({"reps": args.case_steps} if args.case_steps is not None else {}))
    else:
        if args.case_steps:
            kw["steps"] = args.case_steps
        res = measure_fit(nb, inputs, dev, stream, **kw)
    print(json.dumps({"case": args.case, **res}))
    return 0


def measure_paths(nb, inputs, w, params_bf16, dev, stream, peak, reps=200):
    """Per-kernel CUDA-event timings of the comparison paths at the same N."""
    import torch
    N, L = w.n, w.n_lobes
    cam = tuple(float(x) for x in w.cam)
    p32 = torch.from_numpy(w.params).to(dev)
    c32 = torch.from_numpy(w.c0).to(dev)
    c16 = c32.to(torch.bfloat16)
    means = torch.from_numpy(w.means).to(dev)
    g = torch.from_numpy(w.g_rgb).to(dev)
    rgb = torch.empty((N, 3), device=dev)
    gp = torch.empty(p32.shape, device=dev)
    gc = torch.empty((3, N), device=dev)
    gm = torch.empty((N, 3), device=dev)
    coeffs = torch.from_numpy(inputs.sh_coefficients(N, 3, SEED)).to(dev)
    gco = torch.empty_like(coeffs)

    kernels = {
        "nasgabor_fwd_f32": (lambda: nb.nasgabor_eval_fwd(p32, c32, means, cam, L, rgb=rgb, stream=stream),
                             N * bytes_fwd_f32(L)),
        "nasgabor_bwd_f32": (lambda: nb.nasgabor_eval_bwd(p32, means, cam, g, L, g_params=gp, g_c0=gc,
                                                          g_means=gm, stream=stream), N * bytes_bwd_f32(L)),
        "nasgabor_fused_f32": (lambda: nb.nasgabor_fused_fwd_bwd(p32, c32, means, cam, g, L,
                                                                 out=(rgb, gp, gc, gm), stream=stream),
                               N * bytes_fused_f32(L)),
        "nasgabor_fused_bf16": (lambda: nb.nasgabor_fused_fwd_bwd(params_bf16, c16, means, cam, g, L,
                                                                  out=(rgb, gp, gc, gm), stream=stream),
                                N * bytes_fused_bf16(L)),
        "sh3_fwd_f32": (lambda: nb.sh_eval_fwd(coeffs, means, cam, 3, rgb=rgb, stream=stream), N * BYTES_SH3_FWD),
        "sh3_bwd_f32": (lambda: nb.sh_eval_bwd(coeffs, means, cam, g, 3, g_coeffs=gco, g_means=gm,
                                               stream=stream), N * BYTES_SH3_BWD),
    }
    # config 2 through the torch.autograd.Function (what a PyTorch user calls): forward,
    # then .backward of the colours with the upstream gradient; gradients set to None
    # before each pass, as optimizer.zero_grad() does
    p_ag = p32.clone().requires_grad_(True)
    c_ag = c32.clone().requires_grad_(True)
    m_ag = means.clone().requires_grad_(True)

    def autograd_pass():
        p_ag.grad = c_ag.grad = m_ag.grad = None
        nb.NasgEval.apply(p_ag, c_ag, m_ag, cam, L).backward(g)

    kernels["nasgabor_autograd_f32"] = (autograd_pass, N * (bytes_fwd_f32(L) + bytes_bwd_f32(L)))
    res = {}
    for name, (fn, nbytes) in kernels.items():
        for _ in range(5):
            fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps
        gbs = nbytes / (us * 1e-6) / 1e9
        res[name] = {"us": us, "alg_bytes": nbytes, "gbs": gbs, "frac": gbs / peak}
    t_plain = res["nasgabor_fwd_f32"]["us"] + res["nasgabor_bwd_f32"]["us"]
    t_sh = res["sh3_fwd_f32"]["us"] + res["sh3_bwd_f32"]["us"]
    return {
        "kernels": res,
        "plain_f32_fwd_then_bwd": {"value": N * L / (t_plain * 1e-6), "unit": UNIT, "us": t_plain},
        "fused_f32": {"value": N * L / (res["nasgabor_fused_f32"]["us"] * 1e-6), "unit": UNIT},
        "fused_bf16": {"value": N * L / (res["nasgabor_fused_bf16"]["us"] * 1e-6), "unit": UNIT},
        "sh3_fwd_then_bwd": {"value": N / (t_sh * 1e-6), "unit": "primitives/s",
                             "value_basis_lobes": 16 * N / (t_sh * 1e-6), "us": t_sh},
        "autograd_f32": {"value": N * L / (res["nasgabor_autograd_f32"]["us"] * 1e-6), "unit": UNIT,
                         "us": res["nasgabor_autograd_f32"]["us"],
                         "note": "NasgEval.apply(...).backward(g): forward and backward kernels through the "
                                 "torch.autograd.Function, outputs allocated per pass"},
    }


def bytes_step(L, P=10):
    """Fused forward+backward+Adam per visible primitive: per lobe master, m, v read and
    written (3 x 2 x 4 B per scalar) and the bf16 copy written (2 B per scalar); per
    primitive the index (4), mean (12), upstream gradient (12) read, colour written (12),
    c0 master/m/v read and written (3 x 24) and its bf16 copy written (6)."""
    return L * P * (24 + 2) + 4 + 12 + 12 + 12 + 72 + 6


def measure_scene_step(nb, inputs, dev, stream, peak, n=6_000_000, L=8, seed=1003, order="morton"):
    """Scene-scale training step: noisy-shell scene (primitives stored in Morton order of
    their centres), 8 cameras on a ring, per camera the ordered frustum compaction then one
    fused forward+backward+Adam step (BF16 copies of an FP32 master) on the visible
    primitives, all on one stream with no host sync. Beside it, per camera: the same step
    with the upstream gradient formed in the kernel from target colours (MSE loss mode),
    and the unfused path a PyTorch user would write with this library's kernels: the
    backward of the visible primitives (nasgabor_eval_bwd with the index list) into a
    zeroed gradient buffer, torch.optim.Adam(foreach=True) over the parameters, and the
    BF16 copies (note: the dense Adam also advances the moments of primitives that are
    not visible, which the fused step leaves untouched)."""
    import torch
    sc = inputs.shell_scene(n, L, seed, order=order)
    st = nb.TrainState(torch.from_numpy(sc.params).to(dev), torch.from_numpy(sc.c0).to(dev))
    means = torch.from_numpy(sc.means).to(dev)
    del sc.params
    gs = [torch.from_numpy(inputs.ring_upstream(n, j, seed)).to(dev) for j in range(len(sc.cameras))]
    ws = torch.empty(nb.nasg_frustum_workspace_bytes(n), device=dev, dtype=torch.uint8)
    idx = [torch.empty(n, device=dev, dtype=torch.int32) for _ in sc.cameras]
    nvis = [torch.empty(1, device=dev, dtype=torch.int32) for _ in sc.cameras]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * len(sc.cameras) + 1)]
    nc = len(sc.cameras)

    def ring(t0, record, loss="given", upstream=gs):
        for j, cam in enumerate(sc.cameras):
            if record:
                ev[3 * j].record(stream)
            nb.nasg_frustum_compact(means, cam.rot, cam.center, cam.tan_half_fov, idx=idx[j], n_visible=nvis[j],
                                    workspace=ws, stream=stream)
            if record:
                ev[3 * j + 1].record(stream)
            nb.nasgabor_fused_step(st, means, cam.center, upstream[j], L, t0 + j + 1, idx=idx[j],
                                   n_idx_device=nvis[j], stream=stream, loss=loss)
            if record:
                ev[3 * j + 2].record(stream)

    ring(0, False)
    torch.cuda.synchronize(dev)
    ring(nc, True)
    torch.cuda.synchronize(dev)
    vis = [int(v.item()) for v in nvis]
    step_us = [ev[3 * j + 1].elapsed_time(ev[3 * j + 2]) * 1e3 for j in range(nc)]
    comp_us = [ev[3 * j].elapsed_time(ev[3 * j + 1]) * 1e3 for j in range(nc)]
    total_us = ev[0].elapsed_time(ev[3 * nc - 1]) * 1e3
    step_bytes = sum(v * bytes_step(L) for v in vis)
    gbs = step_bytes / (sum(step_us) * 1e-6) / 1e9

    # target-driven step (MSE loss mode): targets U[0, 1]^3 per camera
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    targets = [torch.rand((n, 3), device=dev, generator=gen) for _ in range(nc)]
    ring(2 * nc, False, "mse", targets)
    torch.cuda.synchronize(dev)
    ring(3 * nc, True, "mse", targets)
    torch.cuda.synchronize(dev)
    mse_us = [ev[3 * j + 1].elapsed_time(ev[3 * j + 2]) * 1e3 for j in range(nc)]
    del targets

    # unfused: backward of the visible primitives + torch.optim.Adam(foreach) + BF16 copies
    master = torch.nn.Parameter(st.master.clone())
    c0m = torch.nn.Parameter(st.c0_master.clone())
    pbf, cbf = st.params_bf16, st.c0_bf16
    del st
    master.grad = torch.zeros_like(master)
    c0m.grad = torch.zeros_like(c0m)
    opt = torch.optim.Adam([master, c0m], lr=1e-3, foreach=True)
    uev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * nc)]

    def ring_unfused(record):
        for j in range(nc):
            if record:
                uev[2 * j].record(stream)
            master.grad.zero_()
            c0m.grad.zero_()
            nb.nasgabor_eval_bwd(pbf, means, sc.cameras[j].center, gs[j], L, idx=idx[j][:vis[j]],
                                 g_params=master.grad, g_c0=c0m.grad, want_means=False, stream=stream)
            opt.step()
            with torch.no_grad():
                pbf.copy_(master)
                cbf.copy_(c0m)
            if record:
                uev[2 * j + 1].record(stream)

    with torch.cuda.stream(stream):
        ring_unfused(False)
        torch.cuda.synchronize(dev)
        ring_unfused(True)
        torch.cuda.synchronize(dev)
    unfused_us = [uev[2 * j].elapsed_time(uev[2 * j + 1]) * 1e3 for j in range(nc)]
    del opt, master, c0m
    torch.cuda.empty_cache()
    return {"workload": f"noisy shell N={n} ({order} storage order), L={L}, 8 ring cameras, ~45% visible each, "
                        "BF16 copies of FP32 master",
            "visible_per_camera": vis, "step_us_per_camera": step_us, "compaction_us_per_camera": comp_us,
            "total_us_8_cameras": total_us,
            "value": sum(vis) * L / (total_us * 1e-6), "unit": "visible primitive-lobes/s (incl. compaction)",
            "step_alg_bytes_per_visible_primitive": bytes_step(L), "step_gbs": gbs, "step_frac": gbs / peak,
            "mse_loss_step_us_per_camera": mse_us,
            "unfused_us_per_camera": unfused_us,
            "unfused_note": "nasgabor_eval_bwd (visible list) into zeroed f32 gradients + torch.optim.Adam(foreach=True) "
                            "over all parameters + BF16 copies, per camera (compaction excluded)",
            "fused_speedup_vs_unfused": sum(unfused_us) / sum(step_us)}


def measure_batched(nb, inputs, dev, stream, peak, n_scenes=32, seed=1004, reps=20):
    """Batched persistent launch: 32 scenes, N log-uniform in [5e4, 3e6], L uniform in
    {4, 8, 16}, BF16 parameters, fwd+bwd in one autotuned persistent kernel replayed
    from a CUDA graph."""
    import torch
    sizes = inputs.batched_scene_sizes(n_scenes, seed)
    scenes = [inputs.device_point_cloud(n, L, seed * 100 + j, dev, torch.bfloat16) for j, (n, L) in enumerate(sizes)]
    b = nb.Batch(scenes)
    tune = b.autotune(reps=3, stream=stream)
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream(dev)
    s2.wait_stream(stream)
    with torch.cuda.stream(s2):
        with torch.cuda.graph(g, stream=s2):
            b.run(stream=s2)
    stream.wait_stream(s2)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(torch.cuda.current_stream(dev))
    for _ in range(reps):
        g.replay()
    e1.record(torch.cuda.current_stream(dev))
    e1.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / reps
    alg = sum(n * bytes_fused_bf16(L) for n, L in sizes)
    gbs = alg / (us * 1e-6) / 1e9
    return {"workload": f"{n_scenes} scenes, N log-uniform [5e4, 3e6], L in {{4, 8, 16}}, BF16, one persistent launch "
                        "replayed from a CUDA graph",
            "total_primitives": int(sum(n for n, _ in sizes)), "total_lobes": b.total_lobes, "us": us,
            "value": b.total_lobes / (us * 1e-6), "unit": UNIT, "tuning": tune, "alg_bytes": alg, "gbs": gbs,
            "frac": gbs / peak}


def measure_batched_one(nb, inputs, dev, stream, peak, n_lobes=8, reps=100, seed=77):
    """The batched launch and the single-scene fused kernel on the same work: one BF16 scene of
    8e6 / L primitives x L lobes, the batched launch with the staged dynamic schedule (2 blocks
    per SM, 4 sub-tiles) and with the static one. reps = 0 runs each path once (profiling)."""
    import torch
    L = n_lobes
    n = 8_000_000 // L
    sc = inputs.device_point_cloud(n, L, seed, dev, torch.bfloat16)
    sc["n_lobes"] = L
    b = nb.Batch([dict(sc)], sub_tiles=4)
    cam = tuple(float(x) for x in sc["cam"])
    out = (torch.empty((n, 3), device=dev), torch.empty(sc["params"].shape, device=dev),
           torch.empty((3, n), device=dev), torch.empty((n, 3), device=dev))
    tunings = {"batched_dynamic": nb.NasgBatchTuning(1, 2, 4, 1), "batched_static": nb.NasgBatchTuning(0, 2, 4, 1)}

    def single():
        nb.nasgabor_fused_fwd_bwd(sc["params"], sc["c0"], sc["means"], cam, sc["g_rgb"], L, out=out, stream=stream)

    def batched(t):
        b.tuning = t
        b.run(stream=stream)

    runs = [("single", single)] + [(k, lambda t=t: batched(t)) for k, t in tunings.items()]
    res = {"workload": f"one scene, N={n}, L={L}, BF16, fused fwd+bwd: single-scene kernel and the batched launch",
           "n": n, "n_lobes": L}
    alg = n * bytes_fused_bf16(L)
    for name, f in runs:
        for _ in range(5 if reps else 1):
            f()
        if not reps:
            continue
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            f()
        e1.record(stream)
        e1.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps
        res[name] = {"us": us, "frac": alg / (us * 1e-6) / 1e9 / peak}
    torch.cuda.synchronize(dev)
    res["same_rgb"] = bool(torch.equal(out[0], b.scenes[0]["rgb"]))
    return res


def fit_lr(nb, inputs, step, steps):
    """The fitting workload's rate at a (1-based) step: base 1e-3 times the library's cosine
    schedule factor at iteration step - 1 (Supp. C), started at iteration 47 of 200."""
    start = round(inputs.FIT_SCHEDULE_START * steps / inputs.FIT_STEPS)
    return inputs.FIT_LR * nb.nasg_cosine_lr_factor(step - 1, steps, start)


def measure_fit(nb, inputs, dev, stream, n=2_000_000, ls=16, lt=4, steps=200, n_dirs=64, seed=1005):
    """Fitting loop: a 16-lobe BF16 student (FP32 master, Adam at base rate 1e-3 with the
    cosine schedule) fitted to a 4-lobe FP32 teacher field on the same primitives, 64 random
    view directions per step shared by all primitives, 200 steps of the fused fitting kernel
    (compute-bound)."""
    import torch
    t = inputs.device_point_cloud(n, lt, seed, dev)
    s = inputs.device_point_cloud(n, ls, seed + 1, dev)
    st = nb.TrainState(s["params"], s["c0"])
    dirs = [torch.from_numpy(inputs.fit_directions(k, seed, n_dirs)).to(dev) for k in range(1, steps + 2)]
    ws = torch.empty(int(nb.lib.nasgabor_fit_workspace_bytes()), device=dev, dtype=torch.uint8)
    losses = torch.empty(steps, device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    lrs = [fit_lr(nb, inputs, k + 1, steps) for k in range(steps)]
    e0.record(stream)
    for k in range(steps):
        nb.nasgabor_fit_step(st, t["params"], t["c0"], lt, dirs[k], ls, k + 1, lr=lrs[k], loss=losses[k:k + 1],
                             workspace=ws, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    l = losses.cpu().numpy()
    evals = n * n_dirs * (ls + lt) * steps
    sub = fit_subsample_check(nb, inputs, dev, stream) if n == 2_000_000 and steps == 200 else None
    ceilings = pipe_ceilings(nb)
    counts = profiled_fit_counts()
    fractions = None
    if counts is not None:
        per_s = n * steps / (ms * 1e-3)          # (primitive, step) pairs per second
        fractions = {"mufu_of_measured": counts["mufu_ops_per_prim_step"] * per_s / ceilings["mufu_ex2_per_s"],
                     "xu_pipe_active": counts["xu_pipe_active_pct"] / 100.0,
                     "fma_pipe_active": counts["fma_pipe_active_pct"] / 100.0,
                     "issue_active": counts["issue_active_pct"] / 100.0,
                     "note": "mufu_of_measured: the kernel's MUFU operations per (primitive, step), counted "
                             "in its source (profiles/nasgabor_fit_step_500k_ls16_lt4.md), times this run's "
                             "(primitive, step) rate, over the MUFU ex2 rate the pipe probe measured; "
                             "xu/fma_pipe_active and issue_active: ncu utilisation of the committed capture "
                             "(500k primitives, the same kernel instance)"}
    return {"workload": f"fit N={n}, student L={ls} BF16 (FP32 master), teacher L={lt} FP32, {n_dirs} directions/step, "
                        f"{steps} Adam steps, base lr 1e-3 with the cosine schedule from iteration "
                        f"{round(inputs.FIT_SCHEDULE_START * steps / inputs.FIT_STEPS)}",
            "ms_total": ms, "ms_per_step": ms / steps,
            "loss_first": float(l[0]), "loss_last": float(l[-1]),
            "lobe_evaluations_per_s": evals / (ms * 1e-3), "subsample_final_mse": sub,
            "pipe_ceilings": ceilings, "pipe_fractions": fractions,
            "note": "compute-bound; subsample_final_mse: the same fit on the workload's seeded 20k subsample "
                    "against the stored FP64 oracle fit (BF16 storage emulated; oracle_fp64_storage without it)"}


def pipe_ceilings(nb):
    """Issue rates measured by the library's pipe microbenchmark on this GPU: MUFU ex2
    results per second, FP32 FMA lane-instructions per second (scalar, and packed FP32x2
    counted as one instruction per lane pair)."""
    mufu = nb.nasg_pipe_rate(0)
    ffma2_ops = nb.nasg_pipe_rate(1)
    ffma = nb.nasg_pipe_rate(2)
    return {"mufu_ex2_per_s": mufu, "ffma_scalar_per_s": ffma, "ffma2_flops_pairs_per_s": ffma2_ops,
            "fma_instr_per_s": max(ffma, ffma2_ops / 2)}


def profiled_fit_counts():
    """Per (primitive, step) warp-level pipe instruction counts of the fitting kernel from
    the committed ncu summary, or None when the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", "nasgabor_fit_step_500k_ls16_lt4.md")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if line.startswith("- ") and ":" in line:
                    k, v = line[2:].split(":", 1)
                    kv[k.strip()] = v.strip().strip("`")
        if kv.get("source_sha256_16") != fit_source_hash():
            return None
        return {"mufu_ops_per_prim_step": float(kv["mufu_ops_per_prim_step"]),
                "xu_pipe_active_pct": float(kv["xu_pipe_active_pct"]),
                "fma_pipe_active_pct": float(kv["fma_pipe_active_pct"]),
                "issue_active_pct": float(kv["issue_active_pct"])}
    except Exception:
        return None


def fit_source_hash():
    """Hash of the sources the fitting kernel is compiled from (csrc/nasg_*.cuh, nasg_*.h, nasg_fit.cu)."""
    csrc = os.path.join(ROOT, "paper_2606_09794_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(csrc)):
        if (f.startswith("nasg_") and (f.endswith(".cuh") or f.endswith(".h"))) or f == "nasg_fit.cu":
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def fit_subsample_check(nb, inputs, dev, stream):
    """The fit on the workload's 20,000-primitive subsample (numpy-drawn, as the stored
    oracle fit), and the final MSE at the held-out step-201 directions against the FP64
    oracle's value stored in tests/golden/fit_subsample_20k.json (written by the oracle)."""
    import torch
    path = os.path.join(ROOT, "tests", "golden", "fit_subsample_20k.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        gold = json.load(f)
    wl = gold["workload"]
    tp, tc, sp, sc, _ = inputs.fit_subsample(wl["n"], wl["student_lobes"], wl["teacher_lobes"], wl["seed_teacher"],
                                             wl["seed_student"], wl["sample"], wl["seed_sample"])
    st = nb.TrainState(torch.from_numpy(sp).to(dev), torch.from_numpy(sc).to(dev))
    tpd, tcd = torch.from_numpy(tp).to(dev), torch.from_numpy(tc).to(dev)
    steps = wl["steps"]
    losses = torch.empty(steps + 1, device=dev)
    for k in range(1, steps + 2):
        nb.nasgabor_fit_step(st, tpd, tcd, wl["teacher_lobes"],
                             torch.from_numpy(inputs.fit_directions(k, wl["seed_teacher"])).to(dev),
                             wl["student_lobes"], k, lr=fit_lr(nb, inputs, k, steps), loss=losses[k - 1:k],
                             stream=stream)
    gpu = float(losses[steps].item())
    ref = gold["bf16_storage"]["final_mse"]
    return {"gpu": gpu, "oracle": ref, "rel_diff": abs(gpu - ref) / ref, "oracle_fp64_storage": gold["fp64"]["final_mse"],
            "start": gold["bf16_storage"]["start_mse"], "sample": wl["sample"]}


def measure_frame(nb, inputs, dev, stream, n=1_000_000, L=8, width=1920, height=1080, seed=1006, reps=10):
    """One training frame with a real upstream gradient: NASGabor colours of all
    primitives at the camera (BF16 parameters), compositing into a 1920 x 1080 image,
    the L2 loss gradient against a target image, the compositing backward (dL/dcolour),
    and the fused forward+backward+Adam step driven by that gradient."""
    import numpy as np
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    pc = inputs.device_point_cloud(n, L, seed, dev)
    st = nb.TrainState(pc["params"], pc["c0"])
    means = (torch.rand((n, 3), device=dev, generator=g) * 3.0 - 1.5).contiguous()
    scales = torch.exp(torch.rand((n, 3), device=dev, generator=g) * 2.0 - 5.5)
    quats = torch.randn((n, 4), device=dev, generator=g)
    opacity = torch.rand(n, device=dev, generator=g) * 0.9 + 0.05
    target = torch.rand((height, width, 3), device=dev, generator=g)
    cam_c = (0.0, 0.0, -4.0)
    cam = nb.raster_camera(np.eye(3), cam_c, width, height, 0.5 * width / 0.6)
    r = nb.Raster(n, cam, 1 << 26)
    rgb = torch.empty((n, 3), device=dev)
    scale = 2.0 / target.numel()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]

    def frame(t, record=False):
        if record:
            ev[0].record(stream)
        nb.nasgabor_eval_fwd(st.params_bf16, st.c0_bf16, means, cam_c, L, rgb=rgb, stream=stream)
        if record:
            ev[1].record(stream)
        img, T = r.forward(means, scales, quats, opacity, rgb, stream=stream)
        if record:
            ev[2].record(stream)
        g_img = (img - target).mul_(scale)
        if record:
            ev[3].record(stream)
        gc, _ = r.backward(rgb, T, g_img, stream=stream)
        if record:
            ev[4].record(stream)
        nb.nasgabor_fused_step(st, means, cam_c, gc, L, t, stream=stream)
        if record:
            ev[5].record(stream)

    for t in range(1, 4):
        frame(t)
    torch.cuda.synchronize(dev)
    stages = np.zeros(5)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for t in range(4, 4 + reps):
        frame(t)
    e1.record(stream)
    e1.synchronize()
    total = e0.elapsed_time(e1) / reps
    for t in range(4 + reps, 4 + 2 * reps):
        frame(t, record=True)
        ev[5].synchronize()
        stages += [ev[k].elapsed_time(ev[k + 1]) for k in range(5)]
    stages /= reps
    return {"workload": f"training frame: N={n} primitives, L={L} BF16 lobes, {width}x{height} image, "
                        "colours -> compositing -> L2 loss gradient -> compositing backward -> fused step",
            "ms_per_frame": total, "pairs": r.n_pairs,
            "stage_ms": {"colours": stages[0], "composite_fwd": stages[1], "loss_grad": stages[2],
                         "composite_bwd": stages[3], "fused_step": stages[4]},
            "note": "the compositing forward synchronises once to size its sort"}


if __name__ == "__main__":
    sys.exit(main())
