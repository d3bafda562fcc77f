"""The replica path of bench.py on two ranks over gloo (CPU): per-rank chain
seeds, the whole-job reduction (all evaluations, slowest rank's time), and the
reference arm running on rank 0 only."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2506_19866_gb300 import synth
    w = synth.make("n15_c3_t11")
    seed = bench.rank_seed(w, rank)
    evals, t = bench.combine_ranks(1000 * (rank + 1), 1.5 + rank, dist, "cpu")
    dist.barrier()
    out.put((rank, seed, evals, t))
    dist.destroy_process_group()


def test_two_rank_reduction_and_seeds():
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
    (r0, s0, e0, t0), (r1, s1, e1, t1) = res
    assert (r0, r1) == (0, 1)
    assert s0 != s1                       # independent replicas
    assert e0 == e1 == 3000               # evaluations of both ranks
    assert t0 == t1 == 2.5                # the slowest rank's time


def test_reference_arm_only_on_rank_zero(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload = "n15_c3_t11"

    bench.run_reference(A(), 1)           # a non-zero rank does no work and prints nothing
    assert capsys.readouterr().out == ""
