"""Replicas path of bench.py on the CPU: two gloo ranks combine their timing
and counted work the way the GPU ranks do (the slowest rank's time, the sum of
the work), and the reference arm runs on rank 0 only.  Multi-GPU is replicas
only: independent Markov chains, no collective on the data path."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = bench.combine_ranks(dist, 1.0 + rank, [10.0 * (rank + 1), 3.0], "cpu")
    single = bench.combine_ranks(None, 1.0 + rank, [10.0 * (rank + 1)], "cpu")
    q.put((rank, out, single))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, out, single = q.get(timeout=120)
        res[r] = (out, single)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        out, single = res[r]
        assert out == (2.0, 30.0, 6.0)          # max time, summed counts
        assert single == (1.0 + r, 10.0 * (r + 1))


def test_reference_arm_prints_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload = "atom_nc1"
        steps = 1
        warmup = 1
        gpus = 2

    bench.run_reference(Args, rank=1)
    assert capsys.readouterr().out == ""


def test_config_names_the_replicas():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1901_01047_gb300 import inputs
    cfg = bench.config_of(inputs.WORKLOADS["batched256"], 4)
    assert cfg["parallelism"] == "replicas4" and cfg["workload"] == "batched256"
    assert cfg["schedule"] == "pooled"


def test_schedule_override_keeps_the_workload():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload = "batched256"
        schedule = "lockstep"

    wl = bench.workload_of(Args)
    assert wl.schedule == "lockstep" and wl.walkers == 256 and wl.name == "batched256"
    Args.schedule = None
    assert bench.workload_of(Args).schedule == "pooled"
