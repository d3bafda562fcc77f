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


# ---- the control flow of bench.run_ours on two ranks, library stubbed ---------

class _FakeLib:
    """Stands in for the library binding: every network's chains make 10%
    null moves per sweep; rn_anneal counts one launch."""

    def __init__(self):
        self.seeds, self.launches, self.nets, self.P = [], 0, {}, {}

    def rn_create(self, device, stream):
        return 1

    def rn_destroy(self, ctx):
        pass

    def rn_load_network(self, ctx, src, dst, fast):
        nid = len(self.P)
        self.P[nid] = 3 * len(src) + 3 * len(fast)
        return nid

    def rn_load_timecourse(self, ctx, nid, init, ref, observed, knockout):
        pass

    def rn_init_chains(self, ctx, nid, n, seed):
        self.seeds.append(int(seed))
        self.nets[nid] = np.zeros((n, 3), np.int64)

    def rn_get_chain_state(self, ctx, nid, n):
        return dict(x_cur=np.zeros((n, self.P[nid]), np.int8), counters=self.nets[nid].copy(),
                    step=0)

    def rn_evaluate(self, ctx, nid, x, traj_shape=None):
        n = np.atleast_2d(x).shape[0]
        return np.zeros(n, np.int32), np.zeros((n, *traj_shape), np.uint8)

    def schedule(self, *a, **k):
        return (a, k)

    def rn_prepare_schedule(self, ctx, s, n):
        pass

    def rn_anneal(self, ctx, s, sweeps):
        for c in self.nets.values():
            c[:, 2] += sweeps // 10
        self.launches += 1

    def rn_synchronize(self, ctx):
        pass

    def rn_launch_count(self, ctx):
        return self.launches

    def rn_get_best(self, ctx, nid):
        return np.zeros(self.P[nid], np.int8), 0, 0


class _FakeDev:
    """Stands in for the CUDA device: each step takes 10 ms x (rank + 1)."""

    def __init__(self, rank):
        self.index, self.handle, self.sm_count, self.reduce_device = rank, 0, 152, "cpu"
        self.ms = 10.0 * (rank + 1)
        self.t = 0.0

    def synchronize(self):
        pass

    def flush_l2(self):
        pass

    def event(self):
        self.t += self.ms
        return self.t

    def elapsed_ms(self, a, b):
        return b - a

    def memory_used_gb(self):
        return 0.0

    def peaks(self):
        return {"alu": 88.0, "imad": 64.0, "lds": 1.0}

    def clock_sampler(self):
        class C:
            def start(self):
                pass

            def stop(self):
                return {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "reasons": []}
        return C()


class _CountingDist:
    def __init__(self, dist):
        self.dist, self.barriers = dist, 0
        self.ReduceOp = dist.ReduceOp

    def barrier(self):
        self.barriers += 1
        self.dist.barrier()

    def all_reduce(self, t, op):
        self.dist.all_reduce(t, op=op)


def _run_ours_worker(rank, world, port, out):
    import contextlib
    import io
    import types

    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    args = types.SimpleNamespace(workload="n15_c3_t11", sweeps_per_step=10, steps=3, warmup=3,
                                 screened=False, batch_candidate=None, no_e2e=False,
                                 no_ttt=False, no_early_reject=False, no_sub_records=False,
                                 no_cpu_baseline=False, e2e_steps=1, paper_protocol=False,
                                 screen_gain=False, cpu_seconds=1.0)
    lib, dev = _FakeLib(), _FakeDev(rank)
    counting = _CountingDist(dist)
    real_import = __builtins__["__import__"] if isinstance(__builtins__, dict) else \
        __builtins__.__import__
    buf = io.StringIO()

    def fake_import(name, *a, **k):      # run_ours imports torch.distributed as dist
        if name == "torch.distributed":
            return types.SimpleNamespace(distributed=counting)
        return real_import(name, *a, **k)

    import builtins
    builtins.__import__ = fake_import
    try:
        with contextlib.redirect_stdout(buf):
            bench.run_ours(args, rank, world, rank, R=lib, dev=dev)
    finally:
        builtins.__import__ = real_import
    out.put((rank, buf.getvalue(), lib.seeds, lib.launches, counting.barriers))
    dist.destroy_process_group()


def test_run_ours_two_ranks_control_flow():
    # per-rank chain seeds, barriers around the timed steps, the whole-job value
    # (all ranks' evaluations over the slowest rank's time), one line printed by
    # rank 0 alone, and none of the single-GPU extras at N = 2
    import json
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_run_ours_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, out0, seeds0, l0, b0), (r1, out1, seeds1, l1, b1) = res
    assert out1 == "" and len(out0.strip().splitlines()) == 1
    line = json.loads(out0)
    sys.path.insert(0, ROOT)
    import bench
    from paper_2506_19866_gb300 import synth
    w = synth.make("n15_c3_t11")
    # the first draw is the planted vector (setup), the second the rank's chains
    assert seeds0[:2] == [w.planted_seed, bench.rank_seed(w, 0)]
    assert seeds1 == [w.planted_seed, bench.rank_seed(w, 1)]
    assert b0 == b1 == 2                                  # before and after the timed steps
    evals_per_rank = w.n_chains * 10 * 3 - w.n_chains * 1 * 3
    assert line["value"] == pytest.approx(2 * evals_per_rank / (3 * 0.020))
    assert line["n_gpus"] == 2 and line["steps"] == 3 and line["warmup"] == 3
    assert line["gpu_launches"] == 3
    assert "e2e" in line                                  # rank 0's end-to-end figure
    for k in ("time_to_target", "early_reject", "sub_records", "cpu_baseline"):
        assert k not in line
    assert l1 == 3 + 3                                    # rank 1: warm-up + timed, no e2e
