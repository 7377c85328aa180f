"""The N > 1 launch path of bench.py on the CPU: two ranks over gloo (127.0.0.1).

The method runs replicas only (one independent run per GPU, no data-path collective), so
what the ranks share is host logic: the process-group set-up from the torchrun
environment, the barriers around the timed region, the max over ranks of the timed
duration (the slowest replica sets the whole-job time), and the reference arm, which only
rank 0 runs and prints.
"""
import os
import socket
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup(SimpleNamespace(impl="reference"))
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    t = bench.max_over_ranks(w, 1.5 + rank)          # each replica's own duration
    bench.barrier(w)
    out.put((rank, t))
    dist.destroy_process_group()


def test_two_ranks_share_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 2.5, 1: 2.5}


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1, 3.25) == 3.25
    bench.barrier(1)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    bench.run_reference(SimpleNamespace(workload="droplet_3d_128x64x64", steps=1, warmup=3,
                                        lb_steps=200), 2, 1)
    assert capsys.readouterr().out == ""
