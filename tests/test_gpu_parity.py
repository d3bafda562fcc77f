"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Scores, trajectories, initial vectors and whole annealing trajectories
(x_cur, x_best, objective values and counters of every compared chain) must be
identical: the method is integer, and both sides draw the same Philox words.
"""
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
    # one context per test: rn_anneal advances every network of a context
    h = R.rn_create(0)
    yield h
    R.rn_destroy(h)


def _eval_parity(p, X):
    score, traj = R.rn_evaluate(p.ctx, p.id, X, traj_shape=p.shape)
    for k in range(X.shape[0]):
        y, t = O.objective(p.net, p.tc, X[k], return_traj=True)
        np.testing.assert_array_equal(traj[k], t, err_msg=f"vector {k}")
        assert score[k] == y, f"vector {k}"


@pytest.mark.parametrize("name", synth.WORKLOADS)
def test_evaluate_workloads(ctx, name):
    p = Problem(synth.make(name), ctx)
    X = np.concatenate([p.xs[None], O.init_chains(p.net, 5, 8), random_vectors(p.net, 8, 1)])
    _eval_parity(p, X)
    if p.w.noise_frac == 0:
        assert R.rn_evaluate(ctx, p.id, p.xs)[0] == 0


@pytest.mark.parametrize("n_nodes", [2, 3, 5, 31, 32, 33, 63, 64, 65, 97, 127, 128,
                                     129, 160, 200, 300, 511])
def test_evaluate_sizes(ctx, n_nodes):
    # word and slot boundaries of the lane layout: 1-4 nodes per lane in
    # registers, 5-16 nodes per lane with the shared-memory tables
    w = synth.random_network(100 + n_nodes, n_nodes, lam=3.0, cap=min(9, n_nodes - 1),
                             n_cond=3, n_times=9, obs_frac=0.4)
    p = Problem(w, ctx)
    _eval_parity(p, random_vectors(p.net, 12, n_nodes))


@pytest.mark.parametrize("n_nodes,n_cond", [(150, 1), (300, 5)])
def test_anneal_shared_memory_path(ctx, n_nodes, n_cond):
    # networks above 128 nodes anneal with the shared-memory tables
    w = synth.random_network(7 + n_nodes, n_nodes, lam=4.0, cap=12, n_cond=n_cond, n_times=9,
                             obs_frac=0.3)
    p = Problem(w, ctx)
    n = 600
    R.rn_init_chains(ctx, p.id, n, 5)
    sched = R.schedule(4.0, 0.99)
    R.rn_anneal(ctx, sched, 20)
    R.rn_anneal(ctx, sched, 20)
    st = R.rn_get_chain_state(ctx, p.id, n)
    ids = [0, 1, 31, 32, 299, 598, 599]
    ch = _oracle_run(p, 5, n, O.Schedule(4.0, 0.99), 0, 40, ids)
    _compare(st, ch, ids)


@pytest.mark.parametrize("T", [1, 2, 33])
def test_evaluate_time_lengths(ctx, T):
    w = synth.random_network(7, 40, lam=4.0, cap=12, n_cond=2, n_times=T, obs_frac=0.6)
    p = Problem(w, ctx)
    _eval_parity(p, random_vectors(p.net, 6, T))


@pytest.mark.parametrize("n_nodes,n_cond", [(40, 1), (40, 5), (100, 8), (200, 3), (400, 2),
                                            (700, 3)])
def test_evaluate_longest_time_course(ctx, n_nodes, n_cond):
    # T = 128, the most accepted: drive counters and u * (steps since the last
    # update) take their widest values on every table path (scalar, grouped
    # conditions, shared-memory tables, hybrid, block)
    w = synth.random_network(300 + n_nodes, n_nodes, lam=4.0, cap=12, n_cond=n_cond,
                             n_times=128, obs_frac=0.3)
    p = Problem(w, ctx)
    _eval_parity(p, random_vectors(p.net, 6, n_nodes))


def test_evaluate_high_degree(ctx):
    # in-degree up to 16 (the largest compiled slot capacity)
    w = synth.random_network(9, 60, lam=10.0, cap=16, n_cond=2, n_times=12, obs_frac=0.5)
    p = Problem(w, ctx)
    assert np.bincount(w.dst).max() > 12
    _eval_parity(p, random_vectors(p.net, 8, 2))


def test_evaluate_device_entry(ctx):
    import torch
    p = Problem(synth.make("n120_c8_t21"), ctx)
    X = O.init_chains(p.net, 3, 33)
    xd = torch.from_numpy(X).cuda()
    sd = torch.zeros(33, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    R.rn_evaluate_device(ctx, p.id, 33, xd, sd)
    R.rn_synchronize(ctx)
    expect = [O.objective(p.net, p.tc, x) for x in X]
    np.testing.assert_array_equal(sd.cpu().numpy(), expect)


def test_evaluate_device_refuses_bad_buffers(ctx):
    # host memory, short buffers and tensors of the wrong kind are refused
    # before any launch (the library checks raw addresses against their
    # allocation; the binding checks tensors)
    import torch
    p = Problem(synth.make("n15_c3_t11"), ctx)
    P = p.net.P
    xd = torch.from_numpy(O.init_chains(p.net, 3, 4)).cuda()
    sd = torch.full((4,), -7, dtype=torch.int32, device="cuda")
    host = np.zeros(4 * P, np.int8)
    n0 = R.rn_launch_count(ctx)
    with pytest.raises(R.RNError) as e:
        R.rn_evaluate_device(ctx, p.id, 4, host.ctypes.data, sd.data_ptr())
    assert e.value.code == R.RN_EINVAL and "x_dev" in str(e.value)
    small = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(R.RNError) as e:     # 2^22 vectors of P bytes: past the allocation
        R.rn_evaluate_device(ctx, p.id, 1 << 22, xd.data_ptr(), small.data_ptr())
    assert e.value.code == R.RN_EINVAL and "allocation" in str(e.value)
    for bad in (xd[:3], xd.to(torch.int32), xd.cpu(), xd.t()):
        with pytest.raises(R.RNError) as e:
            R.rn_evaluate_device(ctx, p.id, 4, bad, sd)
        assert e.value.code == R.RN_EINVAL
    R.rn_synchronize(ctx)
    assert R.rn_launch_count(ctx) == n0 and (sd.cpu().numpy() == -7).all()


@pytest.mark.parametrize("name", ["n15_c3_t11", "n120_c8_t21", "mtb_63n_178e"])
def test_init_chains(ctx, name):
    p = Problem(synth.make(name), ctx)
    n = 64
    R.rn_init_chains(ctx, p.id, n, 12345)
    st = R.rn_get_chain_state(ctx, p.id, n)
    X = O.init_chains(p.net, 12345, n)
    np.testing.assert_array_equal(st["x_cur"], X)
    np.testing.assert_array_equal(st["x_best"], X)
    d = np.array([O.objective(p.net, p.tc, x) for x in X])
    np.testing.assert_array_equal(st["d_cur"], d)
    np.testing.assert_array_equal(st["d_best"], d)
    assert st["step"] == 0 and not st["counters"].any()


def _oracle_run(p, seed, n_chains, sched, g0, sweeps, ids=None):
    ids = list(range(n_chains)) if ids is None else list(ids)
    ch = O.start_chains(p.net, p.tc, seed, len(ids), chain_ids=ids)
    O.anneal(p.net, p.tc, sched, seed, ch, g0, sweeps, chain_ids=None if sched.global_sync else ids)
    return ch


def _compare(st, ch, ids):
    np.testing.assert_array_equal(st["x_cur"][ids], ch.x_cur)
    np.testing.assert_array_equal(st["x_best"][ids], ch.x_best)
    np.testing.assert_array_equal(st["d_cur"][ids], ch.d_cur)
    np.testing.assert_array_equal(st["d_best"][ids], ch.d_best)
    np.testing.assert_array_equal(st["counters"][ids, 0], ch.n_accept)
    np.testing.assert_array_equal(st["counters"][ids, 1], ch.n_uphill)
    np.testing.assert_array_equal(st["counters"][ids, 2], ch.n_null)


def test_anneal_small_all_chains(ctx):
    # the 15-node configuration: 64 chains, T0 = 10, alpha = 0.995, every chain compared
    w = synth.make("n15_c3_t11")
    p = Problem(w, ctx)
    R.rn_init_chains(ctx, p.id, w.n_chains, w.chain_seed)
    sched = R.schedule(w.T0, w.alpha)
    # the whole run of the configuration (2000 sweeps, T from 10 down to 4.4e-4),
    # in calls of uneven length, every chain compared at the end
    for k in (300, 200, 1000, 499, 1):
        R.rn_anneal(ctx, sched, k)
    st = R.rn_get_chain_state(ctx, p.id, w.n_chains)
    assert st["step"] == w.sweeps == 2000
    ch = _oracle_run(p, w.chain_seed, w.n_chains, O.Schedule(w.T0, w.alpha), 0, w.sweeps)
    _compare(st, ch, list(range(w.n_chains)))
    x, score, chain = R.rn_get_best(ctx, p.id)
    assert score == int(ch.d_best.min()) and chain == int(np.argmin(ch.d_best))
    np.testing.assert_array_equal(x, ch.x_best[chain])


def test_stats_per_level(ctx):
    # rn_get_stats: the three counters summed over the chains, the chain count
    # and the next step; a level's counts are the difference around its call,
    # equal to the oracle's over every chain
    w = synth.make("n15_c3_t11")
    p = Problem(w, ctx)
    with pytest.raises(R.RNError) as e:
        R.rn_get_stats(ctx, p.id)
    assert e.value.code == R.RN_ESTATE
    R.rn_init_chains(ctx, p.id, w.n_chains, w.chain_seed)
    assert R.rn_get_stats(ctx, p.id) == dict(accepted=0, uphill=0, null=0,
                                            chains=w.n_chains, step=0)
    sched = R.schedule(w.T0, w.alpha, iters_per_level=100)
    osched = O.Schedule(w.T0, w.alpha, iters_per_level=100)
    ch = O.start_chains(p.net, p.tc, w.chain_seed, w.n_chains)
    prev = R.rn_get_stats(ctx, p.id)
    for level in range(3):
        R.rn_anneal(ctx, sched, 100)
        now = R.rn_get_stats(ctx, p.id)
        before = (ch.n_accept.sum(), ch.n_uphill.sum(), ch.n_null.sum())
        O.anneal(p.net, p.tc, osched, w.chain_seed, ch, 100 * level, 100)
        after = (ch.n_accept.sum(), ch.n_uphill.sum(), ch.n_null.sum())
        got = [now[k] - prev[k] for k in ("accepted", "uphill", "null")]
        assert got == [int(a - b) for a, b in zip(after, before)], level
        assert now["step"] == 100 * (level + 1) and now["chains"] == w.n_chains
        prev = now
    st = R.rn_get_chain_state(ctx, p.id, w.n_chains)
    assert [prev[k] for k in ("accepted", "uphill", "null")] == \
        st["counters"].sum(axis=0).tolist()


def test_empty_inputs(ctx):
    # zero vectors to evaluate (host and device entries) and zero sweeps: no
    # work, no launch, the state unchanged
    w = synth.make("n15_c3_t11")
    p = Problem(w, ctx)
    R.rn_init_chains(ctx, p.id, 8, w.chain_seed)
    before = R.rn_get_chain_state(ctx, p.id, 8)
    n0 = R.rn_launch_count(ctx)
    score, traj = R.rn_evaluate(ctx, p.id, np.zeros((0, p.net.P), np.int8), traj_shape=p.shape)
    assert score.shape == (0,) and traj.shape == (0, *p.shape)
    R.rn_evaluate_device(ctx, p.id, 0, None, None)
    R.rn_anneal(ctx, R.schedule(w.T0, w.alpha), 0)
    R.rn_synchronize(ctx)
    assert R.rn_launch_count(ctx) == n0
    after = R.rn_get_chain_state(ctx, p.id, 8)
    for k in ("x_cur", "x_best", "d_cur", "d_best", "counters"):
        np.testing.assert_array_equal(after[k], before[k])
    assert after["step"] == before["step"] == 0


def test_bounded_wait_gives_up_and_reports(ctx):
    # The failure path of the work queue's bounded waits, without any fault: one
    # warp waits (4096 polls) on a counter that nothing advances.  The host reads
    # RN_ETIMEOUT, the flag is cleared, and the context keeps working bit-exactly.
    w = synth.make("n15_c3_t11")
    p = Problem(w, ctx)
    R.rn_init_chains(ctx, p.id, 8, w.chain_seed)
    n0 = R.rn_launch_count(ctx)
    with pytest.raises(R.RNError) as e:
        R.rn_selftest_wait(ctx)
    assert e.value.code == R.RN_ETIMEOUT and "gave up" in str(e.value)
    assert R.rn_launch_count(ctx) == n0 + 1
    R.rn_anneal(ctx, R.schedule(w.T0, w.alpha), 30)
    st = R.rn_get_chain_state(ctx, p.id, 8)
    ch = _oracle_run(p, w.chain_seed, 8, O.Schedule(w.T0, w.alpha), 0, 30)
    _compare(st, ch, list(range(8)))


def test_out_of_memory_is_reported_and_recoverable(ctx):
    # chains far beyond the device's memory (2^31 - 1 rows of 192 bytes): RN_ENOMEM,
    # and the same context keeps working bit-exactly afterwards
    w = synth.make("n15_c3_t11")
    p = Problem(w, ctx)
    with pytest.raises(R.RNError) as e:
        R.rn_init_chains(ctx, p.id, 2 ** 31 - 1, w.chain_seed)
    assert e.value.code == R.RN_ENOMEM
    R.rn_init_chains(ctx, p.id, 8, w.chain_seed)
    R.rn_anneal(ctx, R.schedule(w.T0, w.alpha), 30)
    st = R.rn_get_chain_state(ctx, p.id, 8)
    ch = _oracle_run(p, w.chain_seed, 8, O.Schedule(w.T0, w.alpha), 0, 30)
    _compare(st, ch, list(range(8)))


def test_anneal_large_subset(ctx):
    # the 120-node configuration at its full chain count (4096), 16 chains compared
    w = synth.make("n120_c8_t21")
    p = Problem(w, ctx)
    R.rn_init_chains(ctx, p.id, w.n_chains, w.chain_seed)
    sched = R.schedule(w.T0, w.alpha)
    R.rn_anneal(ctx, sched, 60)
    st = R.rn_get_chain_state(ctx, p.id, w.n_chains)
    ids = [0, 1, 2, 3, 151, 152, 600, 1023, 1024, 2047, 2048, 3000, 4000, 4093, 4094, 4095]
    ch = _oracle_run(p, w.chain_seed, w.n_chains, O.Schedule(w.T0, w.alpha), 0, 60, ids)
    _compare(st, ch, ids)
    # every chain: the stored objective is the objective of the stored vector
    sample = np.arange(0, w.n_chains, 97)
    y = R.rn_evaluate(ctx, p.id, st["x_cur"][sample])
    np.testing.assert_array_equal(y, st["d_cur"][sample])
    assert (st["d_best"] <= st["d_cur"]).all()


def _chains_of(st, ids):
    """The oracle's view of the GPU chains `ids` at a hand-over point."""
    c = st["counters"][ids]
    return O.Chains(st["x_cur"][ids], st["d_cur"][ids], st["x_best"][ids], st["d_best"][ids],
                    c[:, 0], c[:, 1], c[:, 2])


def test_anneal_late_schedule_subset(ctx):
    # The 120-node configuration where its runs spend their time: the GPU
    # anneals all 4096 chains to step 60,000 (T = 0.024) and to step 99,900
    # (T = 4.4e-4, the last 100 steps of the 10^5-step schedule) in 500-step
    # calls from cached threshold tables, as the benchmark does.  At each point
    # 16 chains' state goes to the oracle, and 100 more steps of both sides must
    # agree element by element.  Here every uphill threshold is 0 (empty tables),
    # the level index is large and T is the product of 60,000+ multiplications.
    w = synth.make("n120_c8_t21")
    p = Problem(w, ctx)
    R.rn_init_chains(ctx, p.id, w.n_chains, w.chain_seed)
    sched = R.schedule(w.T0, w.alpha)
    R.rn_prepare_schedule(ctx, sched, w.sweeps)
    osched = O.Schedule(w.T0, w.alpha)
    ids = [0, 5, 77, 151, 600, 1023, 1024, 2047, 2048, 2500, 3000, 3333, 4000, 4093, 4094, 4095]
    g = 0
    for g_check in (60000, 99900):
        while g < g_check:
            k = min(500, g_check - g)
            R.rn_anneal(ctx, sched, k)
            g += k
        st = R.rn_get_chain_state(ctx, p.id, w.n_chains)
        assert st["step"] == g
        assert O.threshold(O.level_temperature(w.T0, w.alpha, g), 1) == 0
        ch = _chains_of(st, ids)
        for k, c in enumerate(ids):    # stored objectives are those of the stored vectors
            assert O.objective(p.net, p.tc, st["x_cur"][c]) == st["d_cur"][c]
            assert O.objective(p.net, p.tc, st["x_best"][c]) == st["d_best"][c]
        O.anneal(p.net, p.tc, osched, w.chain_seed, ch, g, 100, chain_ids=ids)
        R.rn_anneal(ctx, sched, 100)
        g += 100
        after = R.rn_get_chain_state(ctx, p.id, w.n_chains)
        _compare(after, ch, ids)
        moved = (after["counters"][ids, 0] - st["counters"][ids, 0]).sum()
        assert moved > 0          # neutral moves are still accepted this late
    assert g == w.sweeps


def test_anneal_paper_mode_last_levels(ctx):
    # The paper's schedule (T = 1000 -> 0.001 by 0.99, reset to x_best at each
    # level start, global argmin at each level end) near its end: the GPU runs
    # 40 chains to the middle of level 1372, the oracle takes every chain's
    # state there, and both run on across the boundaries into levels 1373 and
    # 1374 to the end of level 1374, the last level above T = 0.001.
    w = synth.make("hpg_9n_25e")
    p = Problem(w, ctx)
    n, iters = 40, 6
    R.rn_init_chains(ctx, p.id, n, 79)
    sched = R.schedule(1000.0, 0.99, iters_per_level=iters, reset_to_best=True,
                       global_sync=True)
    g = 1372 * iters + 2
    R.rn_prepare_schedule(ctx, sched, g + 4 * iters)
    R.rn_anneal(ctx, sched, g - 1000)
    R.rn_anneal(ctx, sched, 1000)
    st = R.rn_get_chain_state(ctx, p.id, n)
    assert st["step"] == g
    assert O.count_levels(1000.0, 1e-3, 0.99) == 1375
    ch = _chains_of(st, list(range(n)))
    k = 1375 * iters - g
    O.anneal(p.net, p.tc, O.Schedule(1000.0, 0.99, iters, True, True), 79, ch, g, k)
    R.rn_anneal(ctx, sched, k)
    after = R.rn_get_chain_state(ctx, p.id, n)
    assert after["step"] == 1375 * iters
    _compare(after, ch, list(range(n)))
    assert (after["d_best"] == after["d_best"][0]).all()    # the last level ended in the argmin


def test_anneal_paper_mode(ctx):
    # Table 1 with levels: reset to x_best and a global argmin at each level end
    w = synth.make("hpg_9n_25e")
    p = Problem(w, ctx)
    n = 40
    R.rn_init_chains(ctx, p.id, n, 77)
    sched = R.schedule(50.0, 0.9, iters_per_level=7, reset_to_best=True, global_sync=True)
    R.rn_anneal(ctx, sched, 25)
    R.rn_anneal(ctx, sched, 24)
    st = R.rn_get_chain_state(ctx, p.id, n)
    ch = _oracle_run(p, 77, n, O.Schedule(50.0, 0.9, 7, True, True), 0, 49)
    _compare(st, ch, list(range(n)))


@pytest.mark.parametrize("group", [1, 6, 40])
def test_anneal_paper_mode_grouped(ctx, group):
    # level-end argmin within groups of consecutive chains (Section 4.5); 40
    # chains in groups of 6 leave a last group of 4
    w = synth.make("hpg_9n_25e")
    p = Problem(w, ctx)
    n = 40
    R.rn_init_chains(ctx, p.id, n, 78)
    sched = R.schedule(50.0, 0.9, iters_per_level=7, reset_to_best=True, global_sync=True,
                       sync_group=group)
    R.rn_anneal(ctx, sched, 25)
    R.rn_anneal(ctx, sched, 24)
    st = R.rn_get_chain_state(ctx, p.id, n)
    ch = _oracle_run(p, 78, n, O.Schedule(50.0, 0.9, 7, True, True, sync_group=group), 0, 49)
    _compare(st, ch, list(range(n)))
    np.testing.assert_array_equal(st["d_best"], ch.d_best)


@pytest.mark.parametrize("n_nodes,n_cond", [(40, 1), (100, 6), (200, 5), (300, 4), (700, 3)])
def test_synchronous_scheme(ctx, n_nodes, n_cond):
    # Section 2.2's synchronous updating (every eligible node moves at every
    # step) on the scalar single-condition path, the register tables, the hybrid
    # path, the shared-memory tables and the block path: evaluated scores and
    # trajectories, and annealing chains (u is not proposed), against the oracle
    w = synth.random_network(80 + n_nodes, n_nodes, lam=4.0, cap=14, n_cond=n_cond, n_times=9,
                             obs_frac=0.3)
    p = Problem(w, ctx, sync=True)
    X = np.concatenate([p.xs[None], random_vectors(p.net, 4, 17)])
    score, traj = R.rn_evaluate(ctx, p.id, X, traj_shape=p.shape)
    for k in range(X.shape[0]):
        y, t = O.objective(p.net, p.tc, X[k], return_traj=True)
        np.testing.assert_array_equal(traj[k], t, err_msg=f"vector {k}")
        assert score[k] == y
    n = 96
    R.rn_init_chains(ctx, p.id, n, 6)
    sched = R.schedule(4.0, 0.98)
    R.rn_anneal(ctx, sched, 30)
    st = R.rn_get_chain_state(ctx, p.id, n)
    ids = [0, 1, 50, 95]
    ch = _oracle_run(p, 6, n, O.Schedule(4.0, 0.98), 0, 30, ids)
    _compare(st, ch, ids)
    E, N = w.E, w.N
    x0 = O.init_chains(p.net, 6, n)
    np.testing.assert_array_equal(st["x_cur"][:, 3 * E:3 * E + N], x0[:, 3 * E:3 * E + N])


def test_synchronous_scheme_in_batch(ctx):
    # a synchronous and a priority network annealed in one batched launch, each
    # against the oracle under its own scheme; switching back restores the
    # priority scheme and its proposals
    ws = [synth.random_network(91, 60, lam=4.0, cap=12, n_cond=4, n_times=8, obs_frac=0.3),
          synth.random_network(92, 150, lam=4.0, cap=12, n_cond=5, n_times=8, obs_frac=0.3)]
    probs = [Problem(ws[0], ctx, sync=True), Problem(ws[1], ctx)]
    for p in probs:
        R.rn_init_chains(ctx, p.id, 64, 8)
    sched = R.schedule(4.0, 0.98)
    R.rn_anneal(ctx, sched, 20)
    assert R.rn_batch_config(ctx)["networks"] == 2
    for p in probs:
        st = R.rn_get_chain_state(ctx, p.id, 64)
        ids = [0, 33, 63]
        ch = _oracle_run(p, 8, 64, O.Schedule(4.0, 0.98), 0, 20, ids)
        _compare(st, ch, ids)
    R.rn_set_update_scheme(ctx, probs[0].id, 0)
    with pytest.raises(R.RNError) as e:
        R.rn_get_best(ctx, probs[0].id)
    assert e.value.code == R.RN_ESTATE
    for bad in ((3, None), (2, None)):     # no such scheme; asynchronous without a selection
        with pytest.raises(R.RNError) as e:
            R.rn_set_update_scheme(ctx, probs[0].id, *bad)
        assert e.value.code == R.RN_EINVAL


def _selection(w, seed):
    rng = np.random.default_rng(seed)
    sel = rng.integers(0, w.N, size=(w.C, w.T)).astype(np.int32)
    sel[rng.random((w.C, w.T)) < 0.1] = -1
    return sel


@pytest.mark.parametrize("n_nodes,n_cond", [(40, 1), (100, 6), (200, 5), (300, 4), (700, 3)])
def test_asynchronous_scheme(ctx, n_nodes, n_cond):
    # Section 2.2's asynchronous updating (one node, drawn for each step, may
    # move) on the single-condition scalar path, the register tables, the hybrid
    # path, the shared-memory tables and the block path: scores, trajectories
    # and chains against the oracle
    w = synth.random_network(60 + n_nodes, n_nodes, lam=4.0, cap=14, n_cond=n_cond, n_times=9,
                             obs_frac=0.3)
    p = Problem(w, ctx, async_sel=_selection(w, n_nodes))
    X = np.concatenate([p.xs[None], random_vectors(p.net, 4, 19)])
    score, traj = R.rn_evaluate(ctx, p.id, X, traj_shape=p.shape)
    for k in range(X.shape[0]):
        y, t = O.objective(p.net, p.tc, X[k], return_traj=True)
        np.testing.assert_array_equal(traj[k], t, err_msg=f"vector {k}")
        assert score[k] == y
    n = 96
    R.rn_init_chains(ctx, p.id, n, 4)
    sched = R.schedule(4.0, 0.98)
    R.rn_anneal(ctx, sched, 30)
    st = R.rn_get_chain_state(ctx, p.id, n)
    ids = [0, 2, 47, 95]
    ch = _oracle_run(p, 4, n, O.Schedule(4.0, 0.98), 0, 30, ids)
    _compare(st, ch, ids)


def test_asynchronous_scheme_in_batch_and_limits(ctx):
    # an asynchronous and a priority network in one batched launch; a node
    # outside the network is refused; a new time course drops the scheme
    ws = [synth.random_network(93, 80, lam=4.0, cap=12, n_cond=4, n_times=8, obs_frac=0.3),
          synth.random_network(94, 150, lam=4.0, cap=12, n_cond=5, n_times=8, obs_frac=0.3)]
    probs = [Problem(ws[0], ctx, async_sel=_selection(ws[0], 1)), Problem(ws[1], ctx)]
    for p in probs:
        R.rn_init_chains(ctx, p.id, 64, 9)
    sched = R.schedule(4.0, 0.98)
    R.rn_anneal(ctx, sched, 20)
    assert R.rn_batch_config(ctx)["networks"] == 2
    for p in probs:
        st = R.rn_get_chain_state(ctx, p.id, 64)
        ids = [0, 31, 63]
        ch = _oracle_run(p, 9, 64, O.Schedule(4.0, 0.98), 0, 20, ids)
        _compare(st, ch, ids)
    bad = _selection(ws[0], 3)
    bad[0, 1] = ws[0].N
    with pytest.raises(R.RNError) as e:
        R.rn_set_update_scheme(ctx, probs[0].id, 2, bad)
    assert e.value.code == R.RN_EINVAL
    p0 = probs[0]
    X = np.concatenate([p0.xs[None], random_vectors(p0.net, 3, 5)])
    np.testing.assert_array_equal(
        R.rn_evaluate(ctx, p0.id, X), [O.objective(p0.net, p0.tc, x) for x in X])
    R.rn_load_timecourse(ctx, p0.id, ws[0].init, p0.tc.ref, ws[0].observed, ws[0].knockout)
    prio = O.Network(ws[0].src, ws[0].dst, ws[0].fast)
    np.testing.assert_array_equal(
        R.rn_evaluate(ctx, p0.id, X), [O.objective(prio, p0.tc, x) for x in X])


def test_scheduling_argument_errors(ctx):
    # out-of-range batch tuning candidates and group sizes are refused
    w = synth.make("hpg_9n_25e")
    p = Problem(w, ctx)
    for bad in (-2, 10):
        with pytest.raises(R.RNError) as e:
            R.rn_batch_tune(ctx, bad)
        assert e.value.code == R.RN_EINVAL
    R.rn_init_chains(ctx, p.id, 8, 1)
    with pytest.raises(R.RNError) as e:
        R.rn_anneal(ctx, R.schedule(5.0, 0.9, iters_per_level=3, global_sync=True,
                                    sync_group=-1), 3)
    assert e.value.code == R.RN_EINVAL


def test_screened_step_under_synchronous_scheme(ctx):
    # the screen's exact simulations use the network's update scheme: with
    # eps = 1 a synchronous network's screened chains equal its plain chains
    w = synth.random_network(96, 90, lam=4.0, cap=12, n_cond=4, n_times=8, obs_frac=0.3)
    p = Problem(w, ctx, sync=True)
    mid, D = R.rn_mlp_create(ctx, p.id, 256, 256, 16)
    rng = np.random.default_rng(2)
    R.rn_mlp_set_weights(ctx, mid, dict(
        W1=(0.05 * rng.standard_normal((D, 256))).astype(np.float32), b1=np.zeros(256, np.float32),
        W2=(0.05 * rng.standard_normal((256, 256))).astype(np.float32),
        b2=np.zeros(256, np.float32), w3=(0.05 * rng.standard_normal(256)).astype(np.float32),
        b3=0.0))
    n = 64
    R.rn_init_chains(ctx, p.id, n, 12)
    sched = R.schedule(5.0, 0.97)
    R.rn_anneal_screened(ctx, mid, sched, 15, K=32, top=2, eps=1.0)
    st = R.rn_get_chain_state(ctx, p.id, n)
    ids = [0, 7, 63]
    ch = _oracle_run(p, 12, n, O.Schedule(5.0, 0.97), 0, 15, ids)
    _compare(st, ch, ids)


def test_checkpoint_resume(ctx):
    w = synth.make("mtb_63n_178e")
    p = Problem(w, ctx)
    n = 96
    sched = R.schedule(5.0, 0.99)
    R.rn_init_chains(ctx, p.id, n, 9)
    R.rn_anneal(ctx, sched, 40)
    saved = R.rn_get_chain_state(ctx, p.id, n)
    R.rn_anneal(ctx, sched, 40)
    straight = R.rn_get_chain_state(ctx, p.id, n)
    ctx2 = R.rn_create(0)
    try:
        q = Problem(w, ctx2)
        R.rn_set_chain_state(ctx2, q.id, 9, saved)
        R.rn_anneal(ctx2, sched, 40)
        resumed = R.rn_get_chain_state(ctx2, q.id, n)
    finally:
        R.rn_destroy(ctx2)
    for k in ("x_cur", "x_best", "d_cur", "d_best", "counters"):
        np.testing.assert_array_equal(resumed[k], straight[k])
    assert resumed["step"] == straight["step"] == 80


def test_frozen_parameters(ctx):
    w = synth.tiny(21, n_nodes=4, indeg=2)
    base = Problem(w, ctx)
    frozen = np.ones(base.net.P, np.uint8)
    frozen[[0, 3, base.net.P - 2]] = 0
    p = Problem(w, ctx, frozen=frozen, frozen_val=base.xs)
    R.rn_init_chains(ctx, p.id, 16, 4)
    R.rn_anneal(ctx, R.schedule(2.0, 0.99), 50)
    st = R.rn_get_chain_state(ctx, p.id, 16)
    ch = _oracle_run(p, 4, 16, O.Schedule(2.0, 0.99), 0, 50)
    _compare(st, ch, list(range(16)))
    # everything fixed: every step is a null move
    q = Problem(w, ctx, frozen=np.ones(base.net.P, np.uint8), frozen_val=base.xs)
    R.rn_init_chains(ctx, q.id, 4, 4)
    R.rn_anneal(ctx, R.schedule(2.0, 0.99), 10)
    st = R.rn_get_chain_state(ctx, q.id, 4)
    assert (st["counters"][:, 2] == 10).all() and not st["counters"][:, :2].any()


def test_rejects_bad_input(ctx):
    w = synth.make("n15_c3_t11")
    with pytest.raises(R.RNError) as e:
        R.rn_load_network(ctx, [0, 1, 1], [1, 0, 1], [0, 0])      # self-loop
    assert e.value.code == R.RN_EINVAL
    with pytest.raises(R.RNError) as e:
        R.rn_load_network(ctx, [0, 0], [1, 1], [0, 0])            # duplicate, node 0 no in-edge
    assert e.value.code == R.RN_EINVAL
    with pytest.raises(R.RNError) as e:
        R.rn_load_network(ctx, [0, 1], [1, 2], [0, 0, 0])         # node 2 has no out-edge
    assert e.value.code == R.RN_EINVAL
    net = R.rn_load_network(ctx, w.src, w.dst, w.fast)
    with pytest.raises(R.RNError) as e:
        R.rn_init_chains(ctx, net, 4, 0)                         # no time course yet
    assert e.value.code == R.RN_ESTATE
    bad_init = w.init.copy()
    bad_init[0, 0] = 3
    with pytest.raises(R.RNError) as e:
        R.rn_load_timecourse(ctx, net, bad_init, np.zeros((w.C, w.T, w.N)), w.observed)
    assert e.value.code == R.RN_EINVAL
    R.rn_load_timecourse(ctx, net, w.init, np.zeros((w.C, w.T, w.N)), w.observed, w.knockout)
    x0 = O.init_chains(O.Network(w.src, w.dst, w.fast), 1, 2)
    x0[1, :w.E] = 0                                             # every weight 0
    with pytest.raises(R.RNError) as e:
        R.rn_init_chains(ctx, net, 2, 0, x0)
    assert e.value.code == R.RN_ECONSTRAINT
    # beyond the block path: more than 4096 nodes
    big = synth.random_network(3, 5000, lam=3.0, cap=8, n_cond=1, n_times=4, obs_frac=0.5)
    bn = R.rn_load_network(ctx, big.src, big.dst, big.fast)
    R.rn_load_timecourse(ctx, bn, big.init, np.zeros((1, 4, 5000)), big.observed)
    with pytest.raises(R.RNError) as e:
        R.rn_init_chains(ctx, bn, 2, 0)
    assert e.value.code == R.RN_EUNSUPPORTED


@pytest.mark.parametrize("n_nodes,n_cond", [(100, 6), (40, 1), (200, 5)])
def test_early_reject_is_exact(ctx, n_nodes, n_cond):
    # register tables with 4 conditions per group, the single-condition scalar
    # update, and the shared-memory tables; at a low temperature most
    # candidates stop early, and the chains must not change at all
    w = synth.random_network(900 + n_nodes, n_nodes, lam=4.0, cap=12, n_cond=n_cond,
                             n_times=13, obs_frac=0.4)
    p = Problem(w, ctx)
    n, sweeps = 300, 40
    runs = []
    for early in (False, True):
        c = R.rn_create(0)
        try:
            q = Problem(w, c)
            R.rn_init_chains(c, q.id, n, 3)
            R.rn_anneal(c, R.schedule(0.3, 0.99, early_reject=early), sweeps)
            runs.append(R.rn_get_chain_state(c, q.id, n))
        finally:
            R.rn_destroy(c)
    for k in ("x_cur", "x_best", "d_cur", "d_best", "counters"):
        np.testing.assert_array_equal(runs[0][k], runs[1][k], err_msg=k)
    ids = [0, 7, 299]
    ch = O.start_chains(p.net, p.tc, 3, n, ids)
    O.anneal(p.net, p.tc, O.Schedule(0.3, 0.99), 3, ch, 0, sweeps, ids)
    np.testing.assert_array_equal(runs[1]["x_cur"][ids], ch.x_cur)
    np.testing.assert_array_equal(runs[1]["d_best"][ids], ch.d_best)
    # the run decides many uphill candidates (rejections), the case that stops early
    cnt = runs[1]["counters"]
    rejected = n * sweeps - cnt[:, 0].sum() - cnt[:, 2].sum()
    assert rejected > n * sweeps // 50


@pytest.mark.parametrize("n_nodes,sync", [(9, False), (20, False), (45, False), (63, True),
                                          (60, False)])
def test_single_condition_four_chains_per_warp(ctx, n_nodes, sync):
    # one condition: with enough chains (at least 12 per SM) four chains share
    # a warp in the byte lanes (1 or 2 nodes per lane); 3651 chains leave the
    # last quad with 3.  Sampled chains of every quad position against the
    # oracle, under the priority and the synchronous scheme; then the same
    # steps with exact early rejection, which keeps one chain per warp, must
    # agree for every chain
    w = synth.random_network(500 + n_nodes, n_nodes, lam=3.0, cap=min(7, n_nodes - 1), n_cond=1,
                             n_times=14, obs_frac=0.5)
    p = Problem(w, ctx, sync=sync)
    n_chains = 3651
    R.rn_init_chains(ctx, p.id, n_chains, 21)
    sched = R.schedule(3.0, 0.98)
    R.rn_anneal(ctx, sched, 17)
    R.rn_anneal(ctx, sched, 23)
    st = R.rn_get_chain_state(ctx, p.id, n_chains)
    ids = [0, 1, 2, 3, 4, 9, 10, 1823, 1824, 2046, 3643, 3646, 3647, 3648, 3649, 3650]
    ch = _oracle_run(p, 21, n_chains, O.Schedule(3.0, 0.98), 0, 40, ids)
    _compare(st, ch, ids)
    R.rn_init_chains(ctx, p.id, n_chains, 21)
    R.rn_anneal(ctx, R.schedule(3.0, 0.98, early_reject=True), 40)
    er = R.rn_get_chain_state(ctx, p.id, n_chains)
    for k in ("x_cur", "x_best", "d_cur", "d_best", "counters"):
        np.testing.assert_array_equal(er[k], st[k], err_msg=k)
