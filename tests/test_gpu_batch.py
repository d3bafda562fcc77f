"""Batched annealing of uneven networks in one persistent launch: every chain of
every network must end bit-identical to annealing that network alone (which
the single-network tests tie to the CPU oracle), through the autotuning trials
and through CUDA-graph replays."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_19866_gb300 import rnanneal as R
from paper_2506_19866_gb300 import synth
from tests.gpu_util import Problem

pytestmark = pytest.mark.gpu


def _batch():
    nets = synth.make_batch(n_nets=7, total_chains=700, seed=11, n_min=8, n_max=300)
    # one more network above 128 nodes (shared-memory tables) and a tiny one
    extra = synth.make_batch(n_nets=2, total_chains=90, seed=3, n_min=200, n_max=260)
    small = synth.make_batch(n_nets=1, total_chains=40, seed=4, n_min=10, n_max=12)
    # one of 129-192 nodes (6 nodes per lane on the hybrid path) and one of
    # 257-320 (10 nodes per lane on the hybrid path of a phased launch)
    mid = synth.make_batch(n_nets=1, total_chains=60, seed=5, n_min=140, n_max=180)
    large = synth.make_batch(n_nets=1, total_chains=50, seed=6, n_min=270, n_max=310)
    nets = nets + extra + small + mid + large
    sizes = [w.N for w in nets]
    assert min(sizes) <= 32 and max(sizes) > 128
    return nets


def _state_all(ctx, probs, nets):
    return [R.rn_get_chain_state(ctx, p.id, w.n_chains) for p, w in zip(probs, nets)]


@pytest.mark.parametrize("pin", [None, 0, 1, 2, 4, 6, 7, 8, 9])
def test_batched_equals_separate_runs(pin):
    # autotuned, and each table-path candidate pinned (1 and 4: the hybrid path
    # for the networks of 129-256 nodes, with 4 and 2 warps per block; 6 and 7:
    # every warp with a large region; 8 and 9: one launch per table path, 9 with
    # the hybrid path)
    from paper_2506_19866_gb300 import build
    build.build()
    nets = _batch()
    sched = R.schedule(6.0, 0.99)
    sweeps = 24
    ctx = R.rn_create(0)
    try:
        probs = [Problem(w, ctx) for w in nets]
        for p, w in zip(probs, nets):
            R.rn_init_chains(ctx, p.id, w.n_chains, w.chain_seed)
        R.rn_prepare_schedule(ctx, sched, 4 * sweeps)
        if pin is not None:
            R.rn_batch_tune(ctx, pin)
        R.rn_anneal(ctx, sched, sweeps)           # tunes (or takes the pinned one), then runs
        cfg = R.rn_batch_config(ctx)
        assert cfg["networks"] == len(nets) and cfg["warps_per_block"] in (2, 4)
        if pin is None:
            assert all(t > 0 for t in cfg["trial_ms"]) and 0 <= cfg["config"] <= 9
        else:
            assert cfg["config"] == pin
            if pin < 8:
                assert cfg["warps_per_block"] == (4 if pin in (0, 1, 2, 6) else 2)
                assert cfg["phases"] == 1
            else:   # one kernel per table path present (at most 1, 2, 4, 6, 8, shared)
                assert 3 <= cfg["phases"] <= 6
            n_hybrid = sum(128 < w.N <= 256 for w in nets)
            assert n_hybrid >= 2
            n_hybrid_phased = sum(128 < w.N <= 320 for w in nets)     # 10 nodes per lane too
            assert cfg["hybrid_networks"] == (n_hybrid if pin in (1, 4) else
                                              n_hybrid_phased if pin == 9 else 0)
        R.rn_anneal(ctx, sched, sweeps)           # graph capture and replay
        R.rn_anneal(ctx, sched, sweeps)
        assert R.rn_batch_config(ctx)["graph"]
        batched = _state_all(ctx, probs, nets)
    finally:
        R.rn_destroy(ctx)
    for p, w, st in zip(probs, nets, batched):
        c1 = R.rn_create(0)
        try:
            q = Problem(w, c1)
            R.rn_init_chains(c1, q.id, w.n_chains, w.chain_seed)
            R.rn_anneal(c1, sched, 3 * sweeps)
            alone = R.rn_get_chain_state(c1, q.id, w.n_chains)
        finally:
            R.rn_destroy(c1)
        for k in ("x_cur", "x_best", "d_cur", "d_best", "counters"):
            np.testing.assert_array_equal(st[k], alone[k], err_msg=f"{w.name} N={w.N} {k}")
        assert st["step"] == alone["step"] == 3 * sweeps


def test_batched_chain_matches_oracle():
    # one chain of the largest network (shared-memory path in the batch)
    from paper_2506_19866_gb300 import build
    build.build()
    nets = _batch()
    big = max(range(len(nets)), key=lambda b: nets[b].N)
    sched = R.schedule(6.0, 0.99)
    ctx = R.rn_create(0)
    try:
        probs = [Problem(w, ctx) for w in nets]
        for p, w in zip(probs, nets):
            R.rn_init_chains(ctx, p.id, w.n_chains, w.chain_seed)
        R.rn_anneal(ctx, sched, 12)
        st = R.rn_get_chain_state(ctx, probs[big].id, nets[big].n_chains)
    finally:
        R.rn_destroy(ctx)
    p, w = probs[big], nets[big]
    ids = [0, w.n_chains - 1]
    ch = O.start_chains(p.net, p.tc, w.chain_seed, len(ids), chain_ids=ids)
    O.anneal(p.net, p.tc, O.Schedule(6.0, 0.99), w.chain_seed, ch, 0, 12, chain_ids=ids)
    np.testing.assert_array_equal(st["x_cur"][ids], ch.x_cur)
    np.testing.assert_array_equal(st["d_best"][ids], ch.d_best)


def test_batched_early_reject_is_exact():
    # the batched launch with exact early rejection: bit-identical chains
    from paper_2506_19866_gb300 import build
    build.build()
    nets = _batch()
    got = []
    for early in (False, True):
        ctx = R.rn_create(0)
        try:
            probs = [Problem(w, ctx) for w in nets]
            for p, w in zip(probs, nets):
                R.rn_init_chains(ctx, p.id, w.n_chains, w.chain_seed)
            R.rn_anneal(ctx, R.schedule(0.4, 0.99, early_reject=early), 20)
            got.append(_state_all(ctx, probs, nets))
        finally:
            R.rn_destroy(ctx)
    for w, a, b in zip(nets, got[0], got[1]):
        for k in ("x_cur", "x_best", "d_cur", "d_best", "counters"):
            np.testing.assert_array_equal(a[k], b[k], err_msg=f"{w.name} {k}")


def test_batch256_full_size_sampled():
    # the 256-network batch (65,536 chains) in the launch configuration the
    # benchmark times: threshold tables cached, the autotuned candidate, the
    # launch replayed from a CUDA graph.  Sampled chains of the smallest, a
    # median, a 129-256-node (hybrid-eligible) and the largest network
    # (shared-memory tables) against the oracle, every field of their state.
    from paper_2506_19866_gb300 import build
    build.build()
    nets = synth.make_batch()
    T0, alpha = nets[0].T0, nets[0].alpha
    sched = R.schedule(T0, alpha)
    S, calls = 8, 3
    order = sorted(range(len(nets)), key=lambda b: nets[b].N)
    picks = [order[0], order[len(order) // 2],
             next(b for b in order if 128 < nets[b].N <= 256), order[-1]]
    ctx = R.rn_create(0)
    try:
        probs = [Problem(w, ctx) for w in nets]
        for p, w in zip(probs, nets):
            R.rn_init_chains(ctx, p.id, w.n_chains, w.chain_seed)
        R.rn_prepare_schedule(ctx, sched, S * calls)
        for _ in range(calls):
            R.rn_anneal(ctx, sched, S)
        cfg = R.rn_batch_config(ctx)
        states = {b: R.rn_get_chain_state(ctx, probs[b].id, nets[b].n_chains) for b in picks}
    finally:
        R.rn_destroy(ctx)
    assert cfg["networks"] == len(nets) and cfg["graph"] and cfg["config"] >= 0
    assert sum(w.n_chains for w in nets) == 65536
    for b in picks:
        p, w, st = probs[b], nets[b], states[b]
        ids = [0, w.n_chains // 2, w.n_chains - 1]
        ch = O.start_chains(p.net, p.tc, w.chain_seed, len(ids), chain_ids=ids)
        O.anneal(p.net, p.tc, O.Schedule(T0, alpha), w.chain_seed, ch, 0, S * calls,
                 chain_ids=ids)
        for k, want in (("x_cur", ch.x_cur), ("x_best", ch.x_best), ("d_cur", ch.d_cur),
                        ("d_best", ch.d_best)):
            np.testing.assert_array_equal(st[k][ids], want, err_msg=f"{w.name} N={w.N} {k}")
        np.testing.assert_array_equal(st["counters"][ids, 0], ch.n_accept)
        np.testing.assert_array_equal(st["counters"][ids, 1], ch.n_uphill)
        np.testing.assert_array_equal(st["counters"][ids, 2], ch.n_null)
