"""Host logic of bench.py's N-process runs, on the CPU.

Two gloo ranks exercise the barrier, the max/sum over ranks and the whole-job
rate (units of all ranks / slowest rank's time); the batched workload's weak
sharding and the reference arm's rank handling are checked without a GPU.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks("gloo")
    r.barrier()
    got = dict(rank=r.rank, world=r.world, mx=r.max(1.0 + rank), sm=r.sum(10.0 * (rank + 1)),
               shard=bench.batched_shard(r.rank, 4),
               rate=bench.whole_job_rate(100.0 * (rank + 1), 1.0 + rank, r))
    r.barrier()
    r.close()
    q.put(got)


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda d: d["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [d["world"] for d in res] == [2, 2]
    for d in res:
        assert d["mx"] == 2.0                      # max over ranks
        assert d["sm"] == 30.0                     # sum over ranks
        assert d["rate"] == pytest.approx(300.0 / 2.0)   # (100 + 200) units / slowest 2 s
    assert res[0]["shard"] == (0, 4) and res[1]["shard"] == (4, 4)


def test_single_process_ranks_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.get(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    for k in env:
        os.environ.pop(k, None)
    try:
        r = bench.Ranks("gloo")
        assert (r.rank, r.world) == (0, 1)
        assert r.max(3.5) == 3.5 and r.sum(2.0) == 2.0
        assert bench.whole_job_rate(10.0, 2.0, r) == 5.0
        r.close()
    finally:
        for k, v in env.items():
            if v is not None:
                os.environ[k] = v


def test_batched_shards_are_disjoint_and_rank0_is_the_single_gpu_batch():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as w
    world = 3
    seq = w.batched_sizes(256 * world, 5)
    got = []
    for r in range(world):
        first, count = bench.batched_shard(r)
        got += w.batched_sizes(count, 5, first=first)
    assert got == seq
    assert w.batched_sizes(256, 5) == seq[:256]


def test_batch_sample_is_bounded():
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    probs = [(9, np.zeros((5, n + 2, n + 2)), None) for n in (1023, 511, 1023, 63, 2047)]
    s, m = bench.batch_sample(probs, budget=1023 ** 2 + 511 ** 2 + 100)
    assert len(s) == 2 and m == 1023 ** 2 + 511 ** 2
    s, m = bench.batch_sample(probs[4:], budget=10)       # always at least one problem
    assert len(s) == 1 and m == 2047 ** 2


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_prints_one_line_small_workload():
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "poisson127", "--steps", "2", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["unit"] == "unknowns/s"
