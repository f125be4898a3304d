"""The benchmark's multi-GPU path is independent replicas (one bed per rank,
no collective on the data path); its host logic runs here as two gloo ranks
on the CPU: the timing is the slowest rank's, the particle count the sum of
all ranks', each rank steps its own seed, and only rank 0 prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch

    sys.path.insert(0, ROOT)
    import bench

    torch.distributed.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                                         world_size=world)
    try:
        ms = bench.reduce_max(10.0 + 5.0 * rank, world, device="cpu")
        n = bench.reduce_sum(1000 * (rank + 1), world, device="cpu")

        class A:
            workload, n, scenes, iters, tol, max_iters, cold, roofline_sweeps, seed, recolour_period = \
                "small", 0, 0, 0, 1e-4, 2000, False, -1, 7, 16
        scene = bench.make_workload(A, rank)
        out.put((rank, ms, n, float(scene["x"][0, 0]), float(scene["x"][5, 1])))
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1] == 15.0          # slowest rank's time
    assert res[0][2] == res[1][2] == 3000.0        # all ranks' particles
    assert res[0][3:] != res[1][3:]                # each rank steps its own seeded bed


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "1",
           "--warmup", "0", "--gpus", "2"]
    r1 = subprocess.run(cmd, cwd=ROOT, env=dict(env, RANK="1", LOCAL_RANK="1"), capture_output=True,
                        text=True, timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = subprocess.run(cmd, cwd=ROOT, env=dict(env, RANK="0", LOCAL_RANK="0"), capture_output=True,
                        text=True, timeout=300)
    assert r0.returncode == 0
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle"
