"""Pins of the CPU oracle to facts outside itself (CPU only).

Each test ties one oracle function to something the paper or mathematics
fixes: hand-derived trajectories and objective values (tests/golden), the
parameter counts the paper prints, closed forms, an independent Philox
implementation, exhaustive search, and invariants.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_19866_gb300 import synth
from tests.helpers import case_network, load_golden, oracle_problem


# ------------------------------------------------------------ Sections 2.1-2.2
@pytest.mark.parametrize("case", load_golden("trajectories.json")["cases"], ids=lambda c: c["name"])
def test_hand_trajectories(case):
    net, x = case_network(case)
    T = case["T"]
    tc = O.Timecourse([case["init"]], np.zeros((1, T, case["n_nodes"])),
                      np.zeros((1, T, case["n_nodes"])), knockout=[case["knockout"]])
    S = O.simulate(net, tc, x, 0)
    np.testing.assert_array_equal(S, np.array(case["S"], dtype=np.uint8), err_msg=case["why"])


# ---------------------------------------------------------------- Section 2.3
@pytest.mark.parametrize("case", load_golden("objective.json")["cases"], ids=lambda c: c["name"])
def test_hand_objective(case):
    N, T = case["n_nodes"], case["T"]
    ref = np.array(case["ref"], np.uint8)
    obs = np.array(case["observed"], np.uint8)
    C = ref.shape[0]
    net = O.Network([0, 1], [1, 0], np.zeros(N, np.uint8))
    tc = O.Timecourse(np.zeros((C, N)), ref, obs)
    np.testing.assert_array_equal(O.weights(net, tc), np.array(case["W"], np.uint8))
    assert O.score_trajectory(net, tc, np.array(case["S"], np.uint8)) == case["y"]
    # with every weight forced to 1 the objective is the unweighted Manhattan distance
    flat_obs = obs.copy()
    flat_obs[:, 1:, :] = 0
    S = np.array(case["S"], np.uint8)
    unweighted = 0
    for t in range(T):
        tc_t = O.Timecourse(np.zeros((C, N)), ref[:, t:t + 1], obs[:, t:t + 1])
        unweighted += O.score_trajectory(net, tc_t, S[:, t:t + 1])
    assert unweighted == case["unweighted"]


def test_objective_zero_iff_match():
    w = synth.tiny(5, n_nodes=4)
    net, tc, xs, _ = oracle_problem(w)
    y, traj = O.objective(net, tc, xs, return_traj=True)
    assert y == 0
    # any single observed mismatch costs exactly its weight times the distance
    W = O.weights(net, tc)
    k = np.flatnonzero(tc.observed.reshape(-1))[0]
    bad = traj.reshape(-1).copy()
    bad[k] = (bad[k] + 1) % 3
    dist = abs(int(bad[k]) - int(tc.ref.reshape(-1)[k]))
    assert O.score_trajectory(net, tc, bad.reshape(traj.shape)) == W.reshape(-1)[k] * dist


# --------------------------------------------- parameter counts (Sections 1, 2.5)
def test_paper_parameter_counts():
    # the paper's two systems: 9 nodes / 25 edges -> 102 parameters and
    # 63 nodes / 178 edges -> 723 parameters, with x = [w, p, t, u, m, d]
    for name, N, E, P in (("hpg_9n_25e", 9, 25, 102), ("mtb_63n_178e", 63, 178, 723)):
        w = synth.make(name)
        assert (w.N, w.E) == (N, E)
        assert O.n_params(O.Network(w.src, w.dst, w.fast)) == P
        assert int(w.observed[0].any(axis=0).sum()) == {102: 5, 723: 35}[P]
        assert w.T == 20


def test_domains():
    net = O.Network([0, 1], [1, 0], np.array([0, 1], np.uint8))
    E, N = 2, 2
    assert list(O.domain(net, 0)) == [0, 1, 2]                  # w
    assert list(O.domain(net, E)) == [-1, 0, 1]                 # p
    assert list(O.domain(net, 2 * E)) == [1, 2]                 # t
    assert list(O.domain(net, 3 * E)) == [1, 2, 3, 4, 5, 6]     # u, slow node
    assert list(O.domain(net, 3 * E + 1)) == [10, 11, 12]       # u, fast node
    assert list(O.domain(net, 3 * E + N)) == [0, 1, 2]          # m
    assert list(O.domain(net, 3 * E + 2 * N)) == [1, 2]         # d


# ------------------------------------------------------ Section 2.4.1 schedule
def test_paper_schedule_levels():
    # T = 1000 down to T_min = 0.001 with rho = 0.99: the number of levels is the
    # smallest n with 1000 * 0.99^n <= 0.001, i.e. ceil(ln(1e-6) / ln(0.99)).
    assert O.count_levels(1000.0, 0.001, 0.99) == math.ceil(math.log(1e-6) / math.log(0.99)) == 1375
    assert O.level_temperature(10.0, 0.995, 0) == 10.0
    assert abs(O.level_temperature(10.0, 0.995, 2000) - 10.0 * 0.995 ** 2000) < 1e-12


# ------------------------------------------------------------------ Philox
def _triton_philox(key, ctrs):
    import os
    os.environ["TRITON_INTERPRET"] = "1"
    # the pin must not pass silently without its reference: a missing Triton
    # fails the test (a chi-square test alone passes a wrong but well-mixed
    # round function)
    try:
        import triton
    except ImportError as e:
        pytest.fail(f"the independent Philox4x32-10 (Triton's interpreter) is unavailable: {e}")
    import torch
    import triton.language as tl

    @triton.jit
    def _k(out_ptr, seed, c0p, c1p, c2p, c3p, n, BLOCK: tl.constexpr):
        offs = tl.arange(0, BLOCK)
        m = offs < n
        a, b, c, d = tl.philox(seed, tl.load(c0p + offs, mask=m), tl.load(c1p + offs, mask=m),
                               tl.load(c2p + offs, mask=m), tl.load(c3p + offs, mask=m))
        tl.store(out_ptr + offs * 4 + 0, a, mask=m)
        tl.store(out_ptr + offs * 4 + 1, b, mask=m)
        tl.store(out_ptr + offs * 4 + 2, c, mask=m)
        tl.store(out_ptr + offs * 4 + 3, d, mask=m)

    n = ctrs.shape[0]
    cols = [torch.from_numpy(np.ascontiguousarray(ctrs[:, k]).view(np.int32)).view(torch.uint32)
            for k in range(4)]
    out = torch.zeros(4 * n, dtype=torch.uint32)
    _k[(1,)](out, key, *cols, n, BLOCK=triton.next_power_of_2(n))
    return out.view(torch.int32).numpy().view(np.uint32).reshape(n, 4)


def test_philox_matches_independent_implementation():
    # Triton's interpreter carries its own Philox4x32-10 (same published round
    # function and constants, written independently); key = (seed_lo, seed_hi).
    rng = np.random.default_rng(7)
    ctrs = rng.integers(0, 2 ** 32, size=(32, 4), dtype=np.uint64).astype(np.uint32)
    ctrs[0] = 0
    ctrs[1] = 0xFFFFFFFF
    for key in (0, 1, 0x123456789ABCDEF, 2 ** 64 - 1):
        ref = _triton_philox(key, ctrs)
        mine = np.stack([O.philox(key, c) for c in ctrs])
        np.testing.assert_array_equal(mine, ref)


def test_philox_uniform_chi2():
    words = np.concatenate([O.philox(0, [g, 0, c, 0]) for g in range(64) for c in range(64)])
    counts = np.bincount((words >> 28).astype(np.int64), minlength=16)
    expected = words.size / 16
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 37.7  # 15 d.o.f., p = 0.001


# ----------------------------------------------------------- Table 1 acceptance
def test_threshold_closed_form_and_bounds():
    for T in (0.01, 0.5, 1.0, 10.0, 1000.0):
        prev = 2 ** 32
        for dE in (1, 2, 3, 5, 10, 50, 200, 1000):
            thr = O.threshold(T, dE)
            assert thr <= prev
            prev = thr
            a = math.exp(-dE / T)
            assert abs(thr / 2 ** 32 - a) <= 2 ** -32 + 1e-15 * a
        # beyond 32 ln 2 * T the acceptance probability is below 2^-32
        assert O.threshold(T, int(32 * math.log(2) * T) + 2) == 0
    # the cap min(., 2^32 - 1): where exp(-dE / T) * 2^32 reaches 2^32 (dE = 0, or
    # dE / T below the double's resolution) the word is the largest, not 0
    assert O.threshold(5.0, 0) == 2 ** 32 - 1
    assert O.threshold(1e20, 1) == 2 ** 32 - 1


def test_metropolis_acceptance_rate():
    # accept iff r < thr with r the third Philox word: for fixed (T, dE) the
    # empirical rate matches exp(-dE / T) within 4 sigma
    n = 20000
    r2 = np.array([O.philox(3, [g, 0, 5, 0])[2] for g in range(n)], dtype=np.uint64)
    for T, dE in ((1.0, 1), (2.0, 3), (10.0, 5), (0.5, 1)):
        p = math.exp(-dE / T)
        rate = float((r2 < O.threshold(T, dE)).mean())
        assert abs(rate - p) < 4 * math.sqrt(p * (1 - p) / n)


# -------------------------------------------------- GetCandidate (Table 1, 2.5.3)
def _constraints_by_definition(src, dst, N, x):
    E = len(src)
    w, p = x[:E], x[E:2 * E]
    out_ok = np.bincount(src[w != 0], minlength=N) >= 1
    in_ok = np.bincount(dst[(w != 0) & (p == 1)], minlength=N) >= 1
    return bool(out_ok.all() and in_ok.all())


def test_propose_is_exactly_the_valid_single_changes():
    w = synth.tiny(3, n_nodes=4, indeg=2)
    net = O.Network(w.src, w.dst, w.fast)
    x = O.init_chain(net, 1, 0)
    n_null = 0
    for k in range(2000):
        r = O.philox(9, [k, 0, 0, 0])
        moved, j, v = O.propose(net, x, r[0], r[1])
        # the alternatives by definition: domain values != x_j whose single
        # change keeps both constraints (Section 2.5.3), ascending
        alts = []
        for val in O.domain(net, j):
            if val == x[j]:
                continue
            y = x.copy()
            y[j] = val
            if _constraints_by_definition(w.src, w.dst, w.N, y):
                alts.append(int(val))
        if moved:
            assert v == alts[(int(r[1]) * len(alts)) >> 32]
            x[j] = v
        else:
            assert alts == []
            n_null += 1
        assert _constraints_by_definition(w.src, w.dst, w.N, x)
    assert n_null > 0  # the walk reaches vectors where some change is blocked
    # index choice: r0 in [k * 2^32 / n, (k+1) * 2^32 / n) picks the k-th free index
    P = net.P
    for k in (0, 1, P // 2, P - 1):
        lo = -(-k * 2 ** 32 // P)
        assert O.propose(net, x, lo, 0)[1] == k
        if k > 0:
            assert O.propose(net, x, lo - 1, 0)[1] == k - 1


def test_propose_respects_frozen():
    w = synth.tiny(4, n_nodes=4, indeg=2)
    net0 = O.Network(w.src, w.dst, w.fast)
    x = O.init_chain(net0, 2, 0)
    frozen = np.ones(net0.P, np.uint8)
    frozen[[1, net0.P - 1]] = 0
    net = O.Network(w.src, w.dst, w.fast, frozen, x)
    seen = set()
    for k in range(200):
        r = O.philox(1, [k, 0, 0, 0])
        moved, j, v = O.propose(net, x, r[0], r[1])
        seen.add(j)
    assert seen == {1, net0.P - 1}


# --------------------------------------------------------- initialisation
def test_init_valid_and_uniform():
    w = synth.make("n120_c8_t21")
    net = O.Network(w.src, w.dst, w.fast)
    X = O.init_chains(net, 0, 200)
    E, N = w.E, w.N
    for x in X:
        assert O.check_params(net, x) == 0
        assert _constraints_by_definition(w.src, w.dst, N, x)
    # t, m, d are never touched by the repair: uniform over their domains
    for lo, hi, k in ((2 * E, 3 * E, 2), (3 * E + N, 3 * E + 2 * N, 3), (3 * E + 2 * N, 3 * E + 3 * N, 2)):
        vals = X[:, lo:hi].reshape(-1)
        counts = np.unique(vals, return_counts=True)[1]
        expected = vals.size / k
        chi2 = float(((counts - expected) ** 2 / expected).sum())
        assert len(counts) == k and chi2 < 16.3  # p = 0.001 at <= 2 d.o.f.
    # distinct chains start from distinct vectors
    assert len({x.tobytes() for x in X}) == len(X)


def _pick(r, n):
    return (int(r) * n) >> 32


def test_init_follows_the_documented_draws():
    # The seeded sample-and-repair sampler as the library documents it, rebuilt
    # from the pinned generator: each x_j = dom_j[pick(word j & 3 of Philox(seed;
    # j >> 2, 0, chain, 1))]; then each node (in order) with no in-edge of p = +1,
    # w != 0 gets the pick(r0)-th of its in-edges set to p = +1, w = 1 + (r1 & 1),
    # r = Philox(seed; i, 0, chain, 3); then each node with no out-edge of w != 0
    # gets the pick(r0)-th of its out-edges set to w = 1 + (r1 & 1), r = Philox(
    # seed; i, 1, chain, 3).  pick(r, n) = floor(r n / 2^32).
    w = synth.tiny(4, n_nodes=6, indeg=2)
    net = O.Network(w.src, w.dst, w.fast)
    E, N, seed = w.E, w.N, 21
    repaired_in = repaired_out = 0
    for chain in range(400):
        x = np.zeros(net.P, np.int8)
        for j in range(net.P):
            dom = O.domain(net, j)
            x[j] = dom[_pick(O.philox(seed, [j >> 2, 0, chain, 1])[j & 3], len(dom))]
        for i in range(N):
            ins = [e for e in range(E) if w.dst[e] == i]
            if any(x[e] != 0 and x[E + e] == 1 for e in ins):
                continue
            r = O.philox(seed, [i, 0, chain, 3])
            e = ins[_pick(r[0], len(ins))]
            x[E + e], x[e] = 1, 1 + (int(r[1]) & 1)
            repaired_in += 1
        for i in range(N):
            outs = [e for e in range(E) if w.src[e] == i]
            if any(x[e] != 0 for e in outs):
                continue
            r = O.philox(seed, [i, 1, chain, 3])
            x[outs[_pick(r[0], len(outs))]] = 1 + (int(r[1]) & 1)
            repaired_out += 1
        np.testing.assert_array_equal(O.init_chain(net, seed, chain), x, err_msg=f"chain {chain}")
    assert repaired_in > 50 and repaired_out > 10


def test_init_reports_unsatisfiable():
    # node 0's only in-edge has p frozen at -1: no activating input is possible
    net = O.Network([1, 0], [0, 1], np.zeros(2, np.uint8),
                    frozen=np.array([0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0], np.uint8),
                    frozen_val=np.array([0, 0, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0], np.int8))
    with pytest.raises(ValueError):
        O.init_chain(net, 0, 0)


# --------------------------------------------------------- simulation invariants
@pytest.mark.parametrize("name", synth.WORKLOADS)
def test_planted_parameters_score_zero(name):
    w = synth.make(name)
    net, tc, xs, flipped = oracle_problem(w)
    y, traj = O.objective(net, tc, xs, return_traj=True)
    if w.noise_frac == 0:
        assert y == 0
    else:
        # every flipped entry costs at most weight 3 times distance 2
        assert 0 < y <= 6 * int(flipped.sum())
    assert traj.max() <= 2
    assert (traj[tc.knockout.astype(bool)[:, None, :].repeat(w.T, axis=1)] == 0).all()
    # deterministic
    assert O.objective(net, tc, xs) == y


# --------------------------------------------------------------- annealing
def _planted_tiny(seed, n_nodes=3, free_frac=0.35):
    w = synth.tiny(seed, n_nodes=n_nodes, indeg=2, n_cond=2, n_times=6, obs_frac=0.7)
    net0, tc, xs, _ = oracle_problem(w, noise=False)
    rng = np.random.default_rng(seed)
    frozen = (rng.random(net0.P) > free_frac).astype(np.uint8)
    net = O.Network(w.src, w.dst, w.fast, frozen, xs)
    return w, net, tc, xs


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bruteforce_optimum_reached_by_anneal(seed):
    w, net, tc, xs = _planted_tiny(seed)
    n_valid, best, bx = O.bruteforce(net, tc)
    assert n_valid >= 1
    assert best == 0  # the planted vector is in the space and scores 0
    # a perturbed target: flip observed entries so the optimum is not 0
    R2, _ = synth.flip_noise(tc.ref, tc.observed, 0.2, seed)
    tc2 = O.Timecourse(tc.init, R2, tc.observed, tc.knockout)
    n2, best2, bx2 = O.bruteforce(net, tc2)
    assert O.objective(net, tc2, bx2) == best2
    sched = O.Schedule(T0=5.0, alpha=0.99)
    ch = O.start_chains(net, tc2, 11, 8)
    O.anneal(net, tc2, sched, 11, ch, 0, 600)
    assert int(ch.d_best.min()) == best2
    for x in ch.x_best:
        assert O.check_params(net, x) == 0


def test_anneal_invariants_and_resume():
    w = synth.tiny(8, n_nodes=5, indeg=2)
    net, tc, xs, _ = oracle_problem(w)
    sched = O.Schedule(T0=3.0, alpha=0.99)
    a = O.start_chains(net, tc, 5, 6)
    O.anneal(net, tc, sched, 5, a, 0, 120)
    for k in range(6):
        assert a.d_cur[k] == O.objective(net, tc, a.x_cur[k])
        assert a.d_best[k] == O.objective(net, tc, a.x_best[k])
        assert a.d_best[k] <= a.d_cur[k]
        assert O.check_params(net, a.x_cur[k]) == 0
        assert a.n_uphill[k] <= a.n_accept[k] and a.n_accept[k] + a.n_null[k] <= 120
    # two calls of 60 steps equal one call of 120 (counter-based generator)
    b = O.start_chains(net, tc, 5, 6)
    O.anneal(net, tc, sched, 5, b, 0, 60)
    O.anneal(net, tc, sched, 5, b, 60, 60)
    np.testing.assert_array_equal(a.x_cur, b.x_cur)
    np.testing.assert_array_equal(a.x_best, b.x_best)
    np.testing.assert_array_equal(a.n_accept, b.n_accept)
    # a subset of chains run alone follows the same trajectories
    ids = [1, 4]
    c = O.start_chains(net, tc, 5, 2, chain_ids=ids)
    O.anneal(net, tc, sched, 5, c, 0, 120, chain_ids=ids)
    np.testing.assert_array_equal(c.x_cur, a.x_cur[ids])
    np.testing.assert_array_equal(c.d_best, a.d_best[ids])


def test_paper_mode_levels():
    w = synth.tiny(9, n_nodes=5, indeg=2)
    net, tc, xs, _ = oracle_problem(w)
    sched = O.Schedule(T0=5.0, alpha=0.9, iters_per_level=10, reset_to_best=True, global_sync=True)
    ch = O.start_chains(net, tc, 2, 5)
    O.anneal(net, tc, sched, 2, ch, 0, 30)
    # after each level every chain holds the global best
    assert len(set(ch.d_best.tolist())) == 1
    assert len({x.tobytes() for x in ch.x_best}) == 1
    assert ch.d_best[0] == O.objective(net, tc, ch.x_best[0])
    # sync requires every chain
    with pytest.raises(RuntimeError):
        O.anneal(net, tc, sched, 2, ch, 30, 10, chain_ids=[0, 1, 2, 3, 4])


def test_synchronous_scheme_closed_form():
    # Section 2.2's synchronous updating with m = 0 and d = 2: every node that is
    # not at its target moves there at once, so each step is the textbook
    # synchronous map S(tau) = clamp(K(S(tau - 1)), 0, 2) node by node, with
    # K_i = sum over in-edges of (s // t) w p (Section 2.1) and knocked-out
    # nodes held at 0.  The priority scheme differs on the same vector.
    w = synth.tiny(21, n_nodes=7, indeg=3, n_cond=3, n_times=9)
    net_s = O.Network(w.src, w.dst, w.fast, sync=True)
    net_p = O.Network(w.src, w.dst, w.fast)
    E, N, C, T = w.E, w.N, w.C, w.T
    tc = O.Timecourse(w.init, np.zeros((C, T, N), np.uint8), w.observed, w.knockout)
    ko = np.zeros((C, N), bool) if w.knockout is None else w.knockout.astype(bool)
    differs = False
    for seed in range(6):
        x = O.init_chain(net_s, 30 + seed, 0).copy()
        x[3 * E + N:3 * E + 2 * N] = 0                  # m = 0
        x[3 * E + 2 * N:] = 2                            # d = 2
        _, S = O.objective(net_s, tc, x, return_traj=True)
        wv, pv, tv = x[:E].astype(int), x[E:2 * E].astype(int), x[2 * E:3 * E].astype(int)
        for c in range(C):
            for tau in range(1, T):
                s = S[c, tau - 1].astype(int)
                K = np.zeros(N, int)
                np.add.at(K, w.dst, (s[w.src] // tv) * wv * pv)
                want = np.clip(K, 0, 2)
                want[ko[c]] = 0
                np.testing.assert_array_equal(S[c, tau], want, err_msg=f"seed {seed} c {c} t {tau}")
        _, Sp = O.objective(net_p, tc, x, return_traj=True)
        differs |= bool((Sp != S).any())
    assert differs
    # the speeds u have no effect, so they are never proposed
    ch = O.start_chains(net_s, tc, 3, 6)
    u0 = ch.x_cur[:, 3 * E:3 * E + N].copy()
    O.anneal(net_s, tc, O.Schedule(5.0, 0.99), 3, ch, 0, 300)
    np.testing.assert_array_equal(ch.x_cur[:, 3 * E:3 * E + N], u0)
    assert (ch.n_accept > 0).all()


def test_asynchronous_scheme_closed_form():
    # Section 2.2's asynchronous updating with the selected node of each step
    # drawn beforehand: with m = 0 and d = 2, at each step only the selected node
    # moves, straight to clamp(K) of the previous states; every other node keeps
    # its state.  Steps whose selection is -1 change nothing.
    w = synth.tiny(22, n_nodes=6, indeg=3, n_cond=2, n_times=12)
    E, N, C, T = w.E, w.N, w.C, w.T
    rng = np.random.default_rng(5)
    sel = rng.integers(0, N, size=(C, T)).astype(np.int32)
    sel[rng.random((C, T)) < 0.15] = -1
    net_a = O.Network(w.src, w.dst, w.fast, async_sel=sel)
    tc = O.Timecourse(w.init, np.zeros((C, T, N), np.uint8), w.observed, w.knockout)
    ko = np.zeros((C, N), bool) if w.knockout is None else w.knockout.astype(bool)
    moved = 0
    for seed in range(5):
        x = O.init_chain(net_a, 40 + seed, 0).copy()
        x[3 * E + N:3 * E + 2 * N] = 0                  # m = 0
        x[3 * E + 2 * N:] = 2                            # d = 2
        _, S = O.objective(net_a, tc, x, return_traj=True)
        wv, pv, tv = x[:E].astype(int), x[E:2 * E].astype(int), x[2 * E:3 * E].astype(int)
        for c in range(C):
            for tau in range(1, T):
                s = S[c, tau - 1].astype(int)
                K = np.zeros(N, int)
                np.add.at(K, w.dst, (s[w.src] // tv) * wv * pv)
                want = s.copy()
                i = sel[c, tau]
                if i >= 0 and not ko[c, i]:
                    want[i] = min(max(K[i], 0), 2)
                np.testing.assert_array_equal(S[c, tau], want, err_msg=f"seed {seed} c {c} t {tau}")
                moved += int((S[c, tau] != S[c, tau - 1]).sum())
    assert moved > 0
    # u has no effect, so it is never proposed
    ch = O.start_chains(net_a, tc, 3, 5)
    u0 = ch.x_cur[:, 3 * E:3 * E + N].copy()
    O.anneal(net_a, tc, O.Schedule(5.0, 0.99), 3, ch, 0, 200)
    np.testing.assert_array_equal(ch.x_cur[:, 3 * E:3 * E + N], u0)


def test_grouped_level_sync():
    # Section 4.5's group-wise reduction: the level-end argmin runs within groups
    # of consecutive chains.  Within a level the chains are independent, so one
    # level with groups of 3 over 7 chains ({0,1,2}, {3,4,5}, {6}) is the plain
    # run followed by each group's argmin (lowest chain on ties) copied into the
    # group's x_best.
    w = synth.tiny(9, n_nodes=5, indeg=2)
    net, tc, xs, _ = oracle_problem(w)
    L, n = 12, 7
    plain = O.start_chains(net, tc, 4, n)
    O.anneal(net, tc, O.Schedule(6.0, 0.9, iters_per_level=L), 4, plain, 0, L)
    grouped = O.start_chains(net, tc, 4, n)
    O.anneal(net, tc, O.Schedule(6.0, 0.9, L, False, True, sync_group=3), 4, grouped, 0, L)
    np.testing.assert_array_equal(grouped.x_cur, plain.x_cur)
    np.testing.assert_array_equal(grouped.d_cur, plain.d_cur)
    for first in range(0, n, 3):
        rows = list(range(first, min(n, first + 3)))
        b = rows[int(np.argmin(plain.d_best[rows]))]   # first index of the minimum
        for k in rows:
            np.testing.assert_array_equal(grouped.x_best[k], plain.x_best[b])
            assert grouped.d_best[k] == plain.d_best[b]
    assert len(set(plain.d_best.tolist())) > 1          # the groups had something to do
    # groups of one chain: no exchange at all, over several levels with resets
    a = O.start_chains(net, tc, 4, n)
    O.anneal(net, tc, O.Schedule(6.0, 0.9, 5, True, True, sync_group=1), 4, a, 0, 40)
    b = O.start_chains(net, tc, 4, n)
    O.anneal(net, tc, O.Schedule(6.0, 0.9, 5, True, False), 4, b, 0, 40)
    np.testing.assert_array_equal(a.x_best, b.x_best)
    np.testing.assert_array_equal(a.x_cur, b.x_cur)
    # one group of at least every chain: the global argmin
    c = O.start_chains(net, tc, 4, n)
    O.anneal(net, tc, O.Schedule(6.0, 0.9, 5, True, True, sync_group=n + 2), 4, c, 0, 40)
    d = O.start_chains(net, tc, 4, n)
    O.anneal(net, tc, O.Schedule(6.0, 0.9, 5, True, True), 4, d, 0, 40)
    np.testing.assert_array_equal(c.x_best, d.x_best)
    np.testing.assert_array_equal(c.x_cur, d.x_cur)
    with pytest.raises(RuntimeError):
        O.anneal(net, tc, O.Schedule(6.0, 0.9, 5, True, True, sync_group=-1), 4, d, 40, 5)


def test_anneal_steps_follow_table1_one_at_a_time():
    # Every step of orc_anneal against Table 1 rebuilt from its parts: r =
    # Philox(seed; g_lo, g_hi, chain, 0) (the pinned generator); GetCandidate on
    # words 0 and 1 (the pinned proposal), a null move when it finds no
    # alternative; accept iff dE <= 0 or word 2 < min(floor(exp(-dE / T_l) 2^32),
    # 2^32 - 1), T_l = T0 alpha^l by repeated multiplication; counters of
    # accepted, accepted uphill (dE > 0) and null moves; x_best on strict
    # improvement only.
    w = synth.tiny(8, n_nodes=5, indeg=2)
    net, tc, xs, _ = oracle_problem(w)
    seed, chain, n_iter, T0, alpha = 13, 3, 7, 4.0, 0.9
    sched = O.Schedule(T0, alpha, iters_per_level=n_iter)
    ch = O.start_chains(net, tc, seed, 1, chain_ids=[chain])
    x, d = ch.x_cur[0].copy(), int(ch.d_cur[0])
    xb, db = x.copy(), d
    n_acc = n_up = n_null = 0
    kinds = set()
    for g in range(400):
        O.anneal(net, tc, sched, seed, ch, g, 1, chain_ids=[chain])
        r = [int(v) for v in O.philox(seed, [g & 0xFFFFFFFF, g >> 32, chain, 0])]
        T = T0
        for _ in range(g // n_iter):
            T *= alpha
        moved, j, v = O.propose(net, x, r[0], r[1])
        if not moved:
            n_null += 1
            kinds.add("null")
        else:
            y = x.copy()
            y[j] = v
            dc = O.objective(net, tc, y)
            dE = dc - d
            accept = dE <= 0 or r[2] < min(math.floor(math.exp(-dE / T) * 2.0 ** 32), 2 ** 32 - 1)
            kinds.add(("down" if dE < 0 else "neutral" if dE == 0 else "up")
                      + ("" if accept else " rejected"))
            if accept:
                x, d = y, dc
                n_acc += 1
                n_up += int(dE > 0)
                if dc < db:
                    xb, db = y.copy(), dc
        np.testing.assert_array_equal(ch.x_cur[0], x, err_msg=f"step {g}")
        np.testing.assert_array_equal(ch.x_best[0], xb, err_msg=f"step {g}")
        assert (int(ch.d_cur[0]), int(ch.d_best[0])) == (d, db), g
        assert (int(ch.n_accept[0]), int(ch.n_uphill[0]), int(ch.n_null[0])) == \
            (n_acc, n_up, n_null), g
    assert {"null", "down", "neutral", "up", "up rejected"} <= kinds


def test_reset_to_best_starts_each_level_from_x_best():
    # reset_to_best (Table 1): each level starts from the chain's x_best.  L
    # levels run with the reset equal the same levels run one at a time without
    # it, with x_cur and delta_cur set to x_best and delta_best by hand first.
    w = synth.tiny(9, n_nodes=5, indeg=2)
    net, tc, xs, _ = oracle_problem(w)
    n, L, n_iter = 5, 6, 8
    a = O.start_chains(net, tc, 7, n)
    O.anneal(net, tc, O.Schedule(6.0, 0.8, n_iter, reset_to_best=True), 7, a, 0, L * n_iter)
    b = O.start_chains(net, tc, 7, n)
    plain = O.Schedule(6.0, 0.8, n_iter)
    away = 0
    for level in range(L):
        away += int((b.x_cur != b.x_best).any())
        b.x_cur[:] = b.x_best
        b.d_cur[:] = b.d_best
        O.anneal(net, tc, plain, 7, b, level * n_iter, n_iter)
    for k in ("x_cur", "x_best", "d_cur", "d_best", "n_accept", "n_uphill", "n_null"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k), err_msg=k)
    assert away > 0                       # some level did start away from x_best


def test_global_argmin_takes_the_lowest_chain_on_ties():
    # The level-end argmin of Table 1 with several chains at the minimum: the
    # lowest chain index wins (the first minimum of a serial scan).  Chains 0-2
    # hold three different vectors that all score 0 on noise-free data of the
    # planted vector; no step can improve on 0, so after one step and the
    # level-end exchange every chain holds chain 0's vector.
    w = synth.tiny(9, n_nodes=5, indeg=2)
    net, tc, xs, _ = oracle_problem(w, noise=False)
    assert O.objective(net, tc, xs) == 0
    zeros = [xs]
    for j in range(net.P):
        for v in O.domain(net, j):
            y = xs.copy()
            y[j] = v
            if v != xs[j] and O.check_params(net, y) == 0 and O.objective(net, tc, y) == 0:
                zeros.append(y)
    assert len(zeros) >= 3
    worse = O.init_chain(net, 5, 0)
    X = np.stack([zeros[1], zeros[2], xs, worse])
    ch = O.Chains(X, np.array([O.objective(net, tc, x) for x in X], np.int32))
    assert list(ch.d_best[:3]) == [0, 0, 0] and ch.d_best[3] > 0
    O.anneal(net, tc, O.Schedule(2.0, 0.9, iters_per_level=1, global_sync=True), 5, ch, 0, 1)
    for k in range(4):
        np.testing.assert_array_equal(ch.x_best[k], zeros[1])
        assert ch.d_best[k] == 0
