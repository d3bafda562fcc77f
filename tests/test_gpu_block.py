"""Block path (513 .. 4096 nodes, a block of 256 threads per chain) against the
CPU oracle through the C ABI: scores and trajectories of evaluated vectors,
and whole annealing chains bit for bit, up to the 2000-node, 16-condition,
33-time-point scale-up network; a batch that mixes a block-path network with
warp-path networks equals separate runs, also with the separate launches on
side streams."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_19866_gb300 import rnanneal as R
from paper_2506_19866_gb300 import synth
from tests.gpu_util import Problem, random_vectors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_2506_19866_gb300 import build
    build.build()


@pytest.fixture
def ctx(built):
    h = R.rn_create(0)
    yield h
    R.rn_destroy(h)


def _compare(st, ch, ids):
    np.testing.assert_array_equal(st["x_cur"][ids], ch.x_cur)
    np.testing.assert_array_equal(st["x_best"][ids], ch.x_best)
    np.testing.assert_array_equal(st["d_cur"][ids], ch.d_cur)
    np.testing.assert_array_equal(st["d_best"][ids], ch.d_best)
    np.testing.assert_array_equal(st["counters"][ids][:, 0], ch.n_accept)
    np.testing.assert_array_equal(st["counters"][ids][:, 1], ch.n_uphill)
    np.testing.assert_array_equal(st["counters"][ids][:, 2], ch.n_null)


@pytest.mark.parametrize("n_nodes,lam,cap,n_cond,n_times", [
    (513, 4.0, 24, 3, 9), (777, 5.0, 24, 5, 7), (1300, 6.0, 24, 2, 12), (600, 20.0, 31, 2, 5),
    (2900, 2.0, 8, 1, 4), (90, 24.0, 31, 3, 6)])
def test_evaluate_block_sizes(ctx, n_nodes, lam, cap, n_cond, n_times):
    # slot and thread boundaries of the block layout (2 .. 12 nodes per thread),
    # one to five conditions (a partial group of 4), in-degrees above the warp
    # paths' 16 (also on a 90-node network, which the block path then takes),
    # and a network near the shared-memory limit; trajectories included
    w = synth.random_network(500 + n_nodes, n_nodes, lam=lam, cap=cap, n_cond=n_cond,
                             n_times=n_times, obs_frac=0.3)
    p = Problem(w, ctx)
    X = np.concatenate([p.xs[None], O.init_chains(p.net, 3, 3), random_vectors(p.net, 3, 9)])
    score, traj = R.rn_evaluate(ctx, p.id, X, traj_shape=p.shape)
    for k in range(X.shape[0]):
        y, t = O.objective(p.net, p.tc, X[k], return_traj=True)
        np.testing.assert_array_equal(traj[k], t, err_msg=f"vector {k}")
        assert score[k] == y, f"vector {k}"
    assert score[0] == 0                        # the planted vector, noise-free data


@pytest.mark.parametrize("seed,n_nodes,lam,cap,n_cond,n_times", [
    (61, 700, 5.0, 20, 6, 8), (64, 1200, 27.0, 31, 2, 5), (65, 2900, 2.0, 8, 1, 4)])
def test_anneal_block_chains_match_oracle(ctx, seed, n_nodes, lam, cap, n_cond, n_times):
    # 700 nodes: node state in registers, x in shared memory; 1200 nodes of
    # in-degree up to 31: the tables leave no room for x, which stays in global
    # memory; 2900 nodes: node state in shared memory (12 nodes per thread)
    w = synth.random_network(seed, n_nodes, lam=lam, cap=cap, n_cond=n_cond, n_times=n_times,
                             obs_frac=0.3)
    p = Problem(w, ctx)
    n = 300                                     # more chains than resident blocks: chunked
    R.rn_init_chains(ctx, p.id, n, 5)
    sched = R.schedule(3.0, 0.98)
    R.rn_anneal(ctx, sched, 10)
    R.rn_anneal(ctx, sched, 14)
    st = R.rn_get_chain_state(ctx, p.id, n)
    assert st["step"] == 24
    ids = [0, 1, 151, 299]
    ch = O.start_chains(p.net, p.tc, 5, n, ids)
    O.anneal(p.net, p.tc, O.Schedule(3.0, 0.98), 5, ch, 0, 24, ids)
    _compare(st, ch, ids)


def test_image_byte_limits(ctx):
    # in-degree 31, the block path's largest: every in-edge of one node
    # activating at full strength (w = 2, p = +1, t = 1, sources in state 2 at
    # t0: K = +124 at the first update) and of another inhibiting (p = -1:
    # K = -124), the extremes one byte of the image holds (evaluation does not
    # require the constraints of Section 2.5.3); in-degree 32 is refused
    w = synth.random_network(66, 600, lam=20.0, cap=31, n_cond=2, n_times=4, obs_frac=0.5)
    indeg = np.bincount(w.dst, minlength=w.N)
    hubs = np.flatnonzero(indeg == 31)[:2]
    assert len(hubs) == 2
    w.init = w.init.copy()
    w.knockout = np.zeros_like(w.knockout)
    for h in hubs:
        w.init[:, w.src[w.dst == h]] = 2
    p = Problem(w, ctx)
    E = w.E
    x = p.xs.copy()
    for h, sign in zip(hubs, (1, -1)):
        e = np.flatnonzero(w.dst == h)
        x[e], x[E + e], x[2 * E + e] = 2, sign, 1
    X = np.stack([x, p.xs])
    score, traj = R.rn_evaluate(ctx, p.id, X, traj_shape=p.shape)
    for k in range(X.shape[0]):
        y, t = O.objective(p.net, p.tc, X[k], return_traj=True)
        np.testing.assert_array_equal(traj[k], t, err_msg=f"vector {k}")
        assert score[k] == y
    over = synth.random_network(67, 600, lam=24.0, cap=32, n_cond=1, n_times=4, obs_frac=0.5)
    assert np.bincount(over.dst, minlength=over.N).max() == 32
    q = Problem(over, ctx)
    with pytest.raises(R.RNError) as e:
        R.rn_init_chains(ctx, q.id, 2, 0)
    assert e.value.code == R.RN_EUNSUPPORTED


@pytest.mark.parametrize("group", [0, 16])
def test_anneal_block_paper_mode(ctx, group):
    # reset to x_best at each level start and the argmin at level end, over all
    # chains or within groups of 16 (the last of 8)
    w = synth.random_network(62, 600, lam=4.0, cap=20, n_cond=2, n_times=6, obs_frac=0.4)
    p = Problem(w, ctx)
    n = 40
    R.rn_init_chains(ctx, p.id, n, 9)
    sched = R.schedule(2.0, 0.9, iters_per_level=5, reset_to_best=True, global_sync=True,
                       sync_group=group)
    R.rn_anneal(ctx, sched, 15)
    st = R.rn_get_chain_state(ctx, p.id, n)
    ids = list(range(n))
    ch = O.start_chains(p.net, p.tc, 9, n)      # the argmin needs every chain
    O.anneal(p.net, p.tc, O.Schedule(2.0, 0.9, 5, True, True, sync_group=group), 9, ch, 0, 15)
    _compare(st, ch, ids)


def test_scale_up_network_sampled(ctx):
    # the 2000-node, 16-condition, 33-time-point network in the launch
    # configuration of a full run (every chain resident): sampled chains and
    # evaluated vectors against the oracle
    w = synth.make("n2000_c16_t33")
    p = Problem(w, ctx)
    n = 2048
    R.rn_init_chains(ctx, p.id, n, w.chain_seed)
    sched = R.schedule(w.T0, w.alpha)
    R.rn_anneal(ctx, sched, 3)
    st = R.rn_get_chain_state(ctx, p.id, n)
    ids = [0, 1777]
    ch = O.start_chains(p.net, p.tc, w.chain_seed, n, ids)
    O.anneal(p.net, p.tc, O.Schedule(w.T0, w.alpha), w.chain_seed, ch, 0, 3, ids)
    _compare(st, ch, ids)
    X = np.concatenate([p.xs[None], st["x_cur"][:2]])
    score = R.rn_evaluate(ctx, p.id, X)
    assert score[0] == 0
    np.testing.assert_array_equal(score[1:], st["d_cur"][:2])


def test_batch_with_block_network_equals_separate_runs(built):
    nets = synth.make_batch(n_nets=3, total_chains=300, seed=21, n_min=20, n_max=200)
    nets.append(synth.random_network(63, 640, lam=4.0, cap=20, n_cond=3, n_times=6,
                                     obs_frac=0.3))
    sched = R.schedule(4.0, 0.97)
    ctx = R.rn_create(0)
    try:
        probs = [Problem(w, ctx) for w in nets]
        for p, w in zip(probs, nets):
            R.rn_init_chains(ctx, p.id, min(w.n_chains, 120), w.chain_seed)
        R.rn_anneal(ctx, sched, 12)
        R.rn_anneal(ctx, sched, 12)
        assert R.rn_batch_config(ctx)["networks"] == 3
        got = [R.rn_get_chain_state(ctx, p.id, min(w.n_chains, 120)) for p, w in zip(probs, nets)]
    finally:
        R.rn_destroy(ctx)
    for w, st in zip(nets, got):
        c1 = R.rn_create(0)
        try:
            q = Problem(w, c1)
            R.rn_init_chains(c1, q.id, min(w.n_chains, 120), w.chain_seed)
            R.rn_anneal(c1, sched, 24)
            alone = R.rn_get_chain_state(c1, q.id, min(w.n_chains, 120))
        finally:
            R.rn_destroy(c1)
        for k in ("x_cur", "x_best", "d_cur", "d_best", "counters"):
            np.testing.assert_array_equal(st[k], alone[k], err_msg=f"{w.name} {k}")


@pytest.mark.parametrize("with_batch", [True, False])
def test_side_stream_launches_equal_separate_runs(built, with_batch):
    # With prepared threshold tables and no global sync, the networks outside
    # the batched launch run on side streams, beside one another and, once the
    # batch is tuned, beside the batched launch.  Three calls: the first tunes
    # the batch (the batch goes first), the next two run in the steady order
    # (side launches first).  The separate networks cover the block path by
    # size and by in-degree, one condition with a warp per chain, and one
    # condition with four chains per warp (24 or more chains per SM, a
    # partial last quad).  Every chain of every network equals that network
    # annealed alone in a context of its own.
    nets, counts = [], []
    if with_batch:
        b = synth.make_batch(n_nets=3, total_chains=300, seed=31, n_min=20, n_max=200)
        nets += b
        counts += [w.n_chains for w in b]
    for w, n in ((synth.random_network(64, 700, lam=4.0, cap=12, n_cond=3, n_times=6,
                                       obs_frac=0.3), 150),
                 (synth.random_network(65, 300, lam=20.0, cap=24, n_cond=2, n_times=5,
                                       obs_frac=0.3), 100),
                 (synth.random_network(66, 40, lam=3.0, cap=8, n_cond=1, n_times=8,
                                       obs_frac=0.4), 200),
                 (synth.random_network(67, 30, lam=3.0, cap=8, n_cond=1, n_times=8,
                                       obs_frac=0.4), 24 * 152 + 5)):
        nets.append(w)
        counts.append(n)
    assert int(np.bincount(nets[-3].dst, minlength=nets[-3].N).max()) > 16
    sched = R.schedule(4.0, 0.97)
    S, calls = 4, 3
    ctx = R.rn_create(0)
    try:
        probs = [Problem(w, ctx) for w in nets]
        for p, w, n in zip(probs, nets, counts):
            R.rn_init_chains(ctx, p.id, n, w.chain_seed)
        R.rn_prepare_schedule(ctx, sched, S * calls)
        for _ in range(calls):
            R.rn_anneal(ctx, sched, S)
        assert R.rn_batch_config(ctx)["networks"] == (3 if with_batch else 0)
        got = [R.rn_get_chain_state(ctx, p.id, n) for p, n in zip(probs, counts)]
    finally:
        R.rn_destroy(ctx)
    for w, n, st in zip(nets, counts, got):
        c1 = R.rn_create(0)
        try:
            q = Problem(w, c1)
            R.rn_init_chains(c1, q.id, n, w.chain_seed)
            R.rn_anneal(c1, sched, S * calls)
            alone = R.rn_get_chain_state(c1, q.id, n)
        finally:
            R.rn_destroy(c1)
        for k in ("x_cur", "x_best", "d_cur", "d_best", "counters"):
            np.testing.assert_array_equal(st[k], alone[k], err_msg=f"{w.name} {k}")


def test_scaleup_full_size_sampled(built):
    # the scale-up set (the 2000-node network with 16,384 chains and 63
    # networks of 100-1000 nodes, 32,768 chains) in the launch configuration
    # the benchmark times: one rn_anneal call runs the batched launch and the
    # block-path launches, threshold tables cached.  Sampled chains of the
    # 2000-node network, a 513-1000-node one, a block-path network by in-degree
    # and the largest and smallest batched networks against the oracle.
    nets = synth.make_scaleup()
    T0, alpha = nets[0].T0, nets[0].alpha
    sched = R.schedule(T0, alpha)
    S, calls = 2, 2
    indeg = [int(np.bincount(w.dst, minlength=w.N).max()) for w in nets]
    blk = [b for b, w in enumerate(nets) if w.N > 512 or indeg[b] > 16]
    warp = [b for b in range(len(nets)) if b not in blk]
    mid = [b for b in blk if 512 < nets[b].N < 2000]
    by_degree = [b for b in blk if nets[b].N <= 512]
    assert nets[0].N == 2000 and mid and by_degree
    picks = [0, mid[0], by_degree[0], max(warp, key=lambda b: nets[b].N),
             min(warp, key=lambda b: nets[b].N)]
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
    assert cfg["networks"] == len(warp)
    assert sum(w.n_chains for w in nets) == 32768
    for b in picks:
        p, w, st = probs[b], nets[b], states[b]
        ids = [0, w.n_chains - 1]
        ch = O.start_chains(p.net, p.tc, w.chain_seed, len(ids), chain_ids=ids)
        O.anneal(p.net, p.tc, O.Schedule(T0, alpha), w.chain_seed, ch, 0, S * calls,
                 chain_ids=ids)
        _compare(st, ch, ids)
