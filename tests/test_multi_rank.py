"""The multi-GPU form is replicas: every rank solves its own copy of the
workload and the benchmark reduces the slowest rank's time and the sum of
candidates.  Covered here with two `gloo` ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 10 ms for 1000 * (r + 1) candidates
        t, c = bench.reduce_over_ranks(10.0 * (rank + 1), 1000.0 * (rank + 1), world, "cpu")
        # every replica runs the same problem list
        names = [(i.name, i.seed, costs) for i, costs in bench.problems()]
        q.put((rank, t, c, names))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_benchmark():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, t, c, names in out:
        assert t == 20.0                  # the slowest rank's time
        assert c == 3000.0                # all ranks' candidates
        assert names == out[0][3]         # replicas: the same workload on every rank
    # whole-job throughput as the benchmark computes it: candidates / slowest time
    assert 3000.0 / (20.0 * 1e-3) == 150000.0


def test_single_rank_needs_no_collective():
    assert bench.reduce_over_ranks(5.0, 7.0, 1, "cpu") == (5.0, 7.0)


def test_reference_arm_prints_only_on_rank_zero(capsys):
    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_arm_runs_the_gpu_arms_problems(capsys):
    """Rank 0 of the reference arm prints one line whose config is the GPU
    arm's (the same 40 problems), with its cpu_baseline and e2e objects."""
    import json

    class A:
        steps, warmup, gpus = 1, 0, 1
    bench.run_reference(A, rank=0, world=1)
    line = json.loads(capsys.readouterr().out)
    assert line["impl"] == "reference"
    assert line["config"] == bench.config_of(1)
    assert line["config"]["problems_per_step"] == 40
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0
