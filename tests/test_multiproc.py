"""The N > 1 path of bench.py on the CPU: world_size-2 gloo ranks.  Multi-GPU here is
replicas only (queries are independent and the index is replicated), so the only cross-rank
work is the max-over-ranks step time and the whole-job rate."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.reduce_max_ms(10.0 + 5.0 * rank, world)
    out[rank] = (ms, bench.replicas_value(1_000_000, ms, world))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, v = out[r]
        assert ms == 15.0
        assert abs(v - 2 * 1_000_000 / 0.015) < 1e-6 * v


def test_reference_arm_other_ranks_exit_quietly(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        config = "small"
        queries = 100
        steps = 1
        warmup = 0
    bench.run_reference(A(), rank=1, world=2)
    assert capsys.readouterr().out == ""
