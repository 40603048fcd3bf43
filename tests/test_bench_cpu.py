"""Host logic of bench.py without a GPU: the multi-rank timing reduction and
shard seeding (world size 2, gloo), the algorithmic byte counts, and the
reference arm's contract line (the FP64 oracle timed on the host)."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    got = bench.reduce_max(10.0 + rank, world)
    q.put((rank, got, bench.shard_seed(bench.SEED, rank)))
    dist.destroy_process_group()


def test_reduce_max_and_shards_over_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]
    assert res[0][2] != res[1][2]


def test_algorithmic_bytes():
    # L = 8: fused BF16 546 B/primitive, plain FP32 fwd+bwd 1044 B/primitive
    assert bench.bytes_fused_bf16(8) == 546
    assert bench.bytes_fwd_f32(8) + bench.bytes_bwd_f32(8) == 1044


def test_reference_arm_prints_contract_line():
    env = dict(os.environ, BENCH_ORACLE_TARGET_S="0.5")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                         timeout=600)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_all_cores_oracle_timing_runs_on_every_core():
    import bench
    r = bench.cpu_oracle_rate_all_cores(target_s=0.2, n_per_proc=200)
    assert r["kind"] == "oracle" and r["value"] > 0
    assert r["cores"] == (os.cpu_count() or 1)
