"""The learned proposal screen on the GPU (through the C ABI) against the FP64
oracle: forward within the derived mixed-precision bound, gradients, training
on pairs the annealer logs, and the screened annealing step (bit-identical to
plain annealing with eps = 1; valid selections and exact scores otherwise)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_19866_gb300 import rnanneal as R
from paper_2506_19866_gb300 import synth
from tests.gpu_util import Problem, random_vectors
from tests.mlp_util import forward_bound, gpu_view, init_weights, spearman, stat_tolerance

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


def _screen(ctx, p, h1, h2, seed, capacity=1 << 16):
    mid, D = R.rn_mlp_create(ctx, p.id, h1, h2, capacity)
    assert D == int(O.onehot_offsets(p.net)[-1])
    params = init_weights(D, h1, h2, p.net.P, seed)
    R.rn_mlp_set_weights(ctx, mid, params)
    return mid, D, params


@pytest.mark.parametrize("name,h1,h2", [("n15_c3_t11", 512, 512), ("mtb_63n_178e", 512, 512),
                                        ("hpg_9n_25e", 256, 768)])
def test_forward_within_bound(ctx, name, h1, h2):
    p = Problem(synth.make(name), ctx)
    mid, D, params = _screen(ctx, p, h1, h2, 11)
    X = random_vectors(p.net, 300, 5)          # 3 row tiles, the last ragged
    y = R.rn_mlp_forward(ctx, mid, X)
    q = gpu_view(params)
    want = O.mlp(p.net, X, q)
    err = np.abs(y.astype(np.float64) - want)
    bound = forward_bound(p.net, X, q)
    tol = stat_tolerance(p.net, X, q)
    print(f"{name}: max error {err.max():.3g}, median 6-sigma tolerance {np.median(tol):.3g}, "
          f"worst-case bound {np.median(bound):.3g}, output std {np.std(want):.3g}")
    assert np.all(err <= bound), f"worst excess {np.max(err - bound)}"
    assert np.all(err <= tol), f"excess over 6 sigma {np.max(err - tol)}"
    # the tolerance means something: well below the spread of the outputs
    assert np.median(tol) < 0.1 * np.std(want)
    # weights round-trip unchanged (FP32 masters)
    back = R.rn_mlp_get_weights(ctx, mid, D, h1, h2)
    for k in ("W1", "b1", "W2", "b2", "w3"):
        np.testing.assert_array_equal(back[k], params[k])
    assert back["b3"] == np.float32(params["b3"])


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("n", [1, 300, 1024])
def test_gradients_match_oracle(ctx, n):
    p = Problem(synth.make("mtb_63n_178e"), ctx)
    h1, h2 = 512, 512
    mid, D, params = _screen(ctx, p, h1, h2, 12)
    X = random_vectors(p.net, n, 6)
    # residuals y - t of a few units, far above the forward error (1e-3), so
    # that dy = 2 (y - t) / n carries no amplified forward error
    rng = np.random.default_rng(7)
    t = (3.0 + rng.standard_normal(n) * 2.0).astype(np.float32)
    loss, g = R.rn_mlp_gradients(ctx, mid, X, t, D, h1, h2)
    y, want_loss, want = O.mlp(p.net, X, gpu_view(params), t)
    rel = {k: _rel(g[k], want[k]) for k in ("W1", "b1", "W2", "b2", "w3", "b3")}
    rel["loss"] = abs(loss - want_loss) / want_loss
    print(f"n={n}: " + ", ".join(f"{k} {v:.2e}" for k, v in rel.items()))
    # the GPU back-propagates BF16-rounded activations and deltas (relative
    # error 2^-8 each) through FP32 accumulation: 1% in norm
    for k, v in rel.items():
        assert v <= 1e-2, k


def test_training_set_ring(ctx):
    p = Problem(synth.make("n15_c3_t11"), ctx)
    mid, _ = R.rn_mlp_create(ctx, p.id, 256, 256, 100)
    X = random_vectors(p.net, 130, 1)
    assert R.rn_mlp_add_samples(ctx, mid, X[:60], np.zeros(60)) == 60
    assert R.rn_mlp_add_samples(ctx, mid, X[60:], np.zeros(70)) == 100
    R.rn_init_chains(ctx, p.id, 40, 3)
    assert R.rn_mlp_log_chains(ctx, mid) == 100
    bad = X[:1].copy()
    bad[0, 0] = 7                                  # w outside {0, 1, 2}
    with pytest.raises(R.RNError):
        R.rn_mlp_forward(ctx, mid, bad)


def _logged_pairs(ctx, p, mid, n_chains, rounds, sweeps, seed):
    """Pairs logged from a plain anneal: every chain's state every `sweeps` steps."""
    R.rn_init_chains(ctx, p.id, n_chains, seed)
    sched = R.schedule(p.w.T0, 0.99)
    for _ in range(rounds):
        R.rn_anneal(ctx, sched, sweeps)
        R.rn_mlp_log_chains(ctx, mid)
    return sched


def test_training_learns_the_score(ctx):
    """Adam on the GPU fits the normalised score y / n_obs of states the annealer
    visits.  Reported on held-out states of an independent run: the global fit
    is weak (the score of a state is a rugged function of 723 parameters; the
    screen's use is ranking single-parameter moves, which the gain test below
    measures), so the stated tolerances are: training loss at least halved,
    held-out Spearman rank correlation >= 0.3, held-out RMSE <= 1.25 x the
    spread of the held-out targets."""
    w = synth.make("mtb_63n_178e")
    p = Problem(w, ctx)
    mid, D = R.rn_mlp_create(ctx, p.id, 512, 512, 1 << 18)
    params = init_weights(D, 512, 512, p.net.P, 13)
    params["W1"] *= 0.5
    R.rn_mlp_set_weights(ctx, mid, params)
    _logged_pairs(ctx, p, mid, 4096, 50, 4, 21)
    first = R.rn_mlp_train(ctx, mid, 1, batch=4096, lr=1e-3, seed=5)
    last = R.rn_mlp_train(ctx, mid, 600, batch=4096, lr=1e-3, seed=6)
    R.rn_init_chains(ctx, p.id, 512, 99)
    R.rn_anneal(ctx, R.schedule(p.w.T0, 0.99), 60)
    st = R.rn_get_chain_state(ctx, p.id, 512)
    n_obs = int(w.observed.sum())
    y_true = st["d_cur"] / n_obs
    y_hat = R.rn_mlp_forward(ctx, mid, st["x_cur"])
    rmse = float(np.sqrt(np.mean((y_hat - y_true) ** 2)))
    rho = spearman(y_hat, y_true)
    print(f"loss {first:.5f} -> {last:.5f}; held-out RMSE {rmse:.4f} (std "
          f"{np.std(y_true):.4f}, mean bias {np.mean(y_hat - y_true):+.4f}), Spearman {rho:.3f}")
    assert last < 0.5 * first
    assert rho >= 0.3
    assert rmse <= 1.25 * np.std(y_true)


def test_training_graph_replay_equals_single_steps(ctx):
    """A training call runs its first Adam step directly and replays the next
    ones from a CUDA graph, the step index and the bias corrections read on the
    device.  With one pair in the training set every minibatch is that pair
    whatever the draw, so k steps in one call must equal k calls of one step
    (which never replay a graph) bit for bit; Adam's step count runs on across
    calls in both."""
    p = Problem(synth.make("n15_c3_t11"), ctx)
    X = random_vectors(p.net, 1, 4)
    screens = []
    for _ in range(2):
        mid, D, params = _screen(ctx, p, 256, 256, 17, capacity=4)
        assert R.rn_mlp_add_samples(ctx, mid, X, np.array([0.3])) == 1
        screens.append(mid)
    before = float(R.rn_mlp_forward(ctx, screens[0], X)[0])
    R.rn_mlp_train(ctx, screens[0], 6, batch=256, lr=1e-3, seed=2)
    for _ in range(6):
        R.rn_mlp_train(ctx, screens[1], 1, batch=256, lr=1e-3, seed=2)
    wa = R.rn_mlp_get_weights(ctx, screens[0], D, 256, 256)
    wb = R.rn_mlp_get_weights(ctx, screens[1], D, 256, 256)
    for k in wa:
        assert np.array_equal(wa[k], wb[k]), k
    assert not np.array_equal(wa["W2"], params["W2"])   # the steps moved the weights
    # towards the one target
    after = float(R.rn_mlp_forward(ctx, screens[0], X)[0])
    assert abs(after - 0.3) < abs(before - 0.3)


def test_screened_eps1_is_plain_annealing(ctx):
    """With eps = 1 every step simulates only candidate 0, the plain proposal:
    chains are bit-identical to rn_anneal's (and so to the oracle's)."""
    w = synth.make("hpg_9n_25e")
    n, sweeps = 256, 60
    sched = R.schedule(10.0, 0.97)
    p = Problem(w, ctx)
    mid, D, _ = _screen(ctx, p, 256, 256, 3)
    R.rn_init_chains(ctx, p.id, n, 17)
    R.rn_anneal_screened(ctx, mid, sched, 25, K=32, top=2, eps=1.0)
    R.rn_anneal_screened(ctx, mid, sched, sweeps - 25, K=32, top=2, eps=1.0)
    st = R.rn_get_chain_state(ctx, p.id, n)
    ctx2 = R.rn_create(0)
    try:
        p2 = Problem(w, ctx2)
        R.rn_init_chains(ctx2, p2.id, n, 17)
        R.rn_anneal(ctx2, sched, sweeps)
        ref = R.rn_get_chain_state(ctx2, p2.id, n)
    finally:
        R.rn_destroy(ctx2)
    for k in ("x_cur", "d_cur", "x_best", "d_best", "counters"):
        np.testing.assert_array_equal(st[k], ref[k], err_msg=k)
    assert st["step"] == ref["step"] == sweeps
    ids = [0, 1, 255]
    ch = O.start_chains(p.net, p.tc, 17, n, ids)
    O.anneal(p.net, p.tc, O.Schedule(10.0, 0.97), 17, ch, 0, sweeps, ids)
    np.testing.assert_array_equal(st["x_cur"][ids], ch.x_cur)
    np.testing.assert_array_equal(st["d_best"][ids], ch.d_best)


@pytest.mark.parametrize("name,h,K", [("mtb_63n_178e", 512, 32), ("n120_c8_t21", 512, 7),
                                      ("n15_c3_t11", 256, 32)])
def test_hidden_rows_in_gemm_equal_through_memory(built, name, h, K):
    """The screened step's two ways of forming the layer-2 input rows -- inside
    the tcgen05 GEMM from A1 and gathered W1 rows (mode 0), or written to memory
    by the propose kernel and read back by TMA (mode 1) -- give the same BF16
    rows and the same MMAs, so the chains come out bit-identical.  301 chains:
    the last row tile is partly padding; K = 7 puts chains across tile edges."""
    w = synth.make(name)
    n, steps = 301, 6
    states = []
    for mode in (0, 1):
        c = R.rn_create(0)
        try:
            p = Problem(w, c)
            mid, D, _ = _screen(c, p, h, h, 9)
            R.rn_mlp_set_hidden_mode(c, mid, mode)
            R.rn_init_chains(c, p.id, n, 5)
            R.rn_anneal_screened(c, mid, R.schedule(2.0, 0.97), steps, K=K, top=2, eps=0.0)
            states.append(R.rn_get_chain_state(c, p.id, n))
            with pytest.raises(R.RNError) as e:
                R.rn_mlp_set_hidden_mode(c, mid, 2)
            assert e.value.code == R.RN_EINVAL
        finally:
            R.rn_destroy(c)
    for k in ("x_cur", "d_cur", "x_best", "d_best", "counters"):
        np.testing.assert_array_equal(states[0][k], states[1][k], err_msg=k)
    assert states[0]["counters"][:, 0].sum() > 0


def _candidates(net, x, seed, chain, g, K):
    """The K candidate moves of step g (oracle GetCandidate on the Philox words)."""
    out = []
    for k in range(K):
        tag = 0 if k == 0 else 16 + k
        r = O.philox(seed, [g & 0xFFFFFFFF, g >> 32, chain, tag])
        ok, j, v = O.propose(net, x, r[0], r[1])
        out.append((j, v) if ok else None)
    return out


@pytest.mark.parametrize("top", [1, 2])
@pytest.mark.parametrize("name,n", [("n15_c3_t11", 96), ("mtb_63n_178e", 97)])
def test_screened_step_selection(ctx, top, name, n):
    """One greedy screened step (T ~ 0, eps = 0): a moved chain took a move that
    can be among the `top` best predicted (oracle prediction +- the derived
    bound) with exact dE <= 0; a chain that stayed had no candidate that is
    surely among them with dE <= 0.  Exact scores are the oracle's.  The
    single-condition network's finish simulates two chains' moves per warp in
    the byte lanes; 97 chains leave the last warp one chain."""
    w = synth.make(name)
    p = Problem(w, ctx)
    h1 = h2 = 256
    mid, D, params = _screen(ctx, p, h1, h2, 4)
    K, seed, g = 32, 23, 0
    R.rn_init_chains(ctx, p.id, n, seed)
    st0 = R.rn_get_chain_state(ctx, p.id, n)
    R.rn_anneal_screened(ctx, mid, R.schedule(1e-9, 1.0), 1, K=K, top=top, eps=0.0)
    st1 = R.rn_get_chain_state(ctx, p.id, n)
    q = gpu_view(params)
    moved = 0
    for c in range(n):
        x0 = st0["x_cur"][c]
        d0 = int(st0["d_cur"][c])
        moves = [m for m in dict.fromkeys(_candidates(p.net, x0, seed, c, g, K)) if m]
        vecs = []
        for j, v in moves:
            xv = x0.copy()
            xv[j] = v
            vecs.append(xv)
        V = np.array(vecs)
        yp = O.mlp(p.net, V, q)
        b = forward_bound(p.net, V, q)
        dE = np.array([O.objective(p.net, p.tc, xv) for xv in V]) - d0
        lo, hi = yp - b, yp + b
        surely_beats = lo[None, :] > hi[:, None]     # [i, k]: i surely ranks before k
        may_beat = lo[:, None] <= hi[None, :]        # [i, k]: i may rank before k
        np.fill_diagonal(may_beat, False)
        possible = surely_beats.sum(axis=0) < top
        sure = may_beat.sum(axis=0) < top
        x1 = st1["x_cur"][c]
        diff = np.flatnonzero(x1 != x0)
        assert len(diff) <= 1
        if len(diff) == 1:
            moved += 1
            k = moves.index((int(diff[0]), int(x1[diff[0]])))
            assert possible[k] and dE[k] <= 0
            assert st1["d_cur"][c] == d0 + dE[k]
            assert st1["counters"][c][0] == 1
        else:
            assert not np.any(sure & (dE <= 0)), f"chain {c}"
            assert st1["d_cur"][c] == d0
    assert moved > n // 4


def test_screened_anneal_invariants(ctx):
    """eps = 0 run: every chain's x_cur keeps the constraints, its stored score
    is exact, x_best holds delta_best, counters add up."""
    w = synth.make("mtb_63n_178e")
    p = Problem(w, ctx)
    mid, D, _ = _screen(ctx, p, 512, 512, 8)
    n = 200
    R.rn_init_chains(ctx, p.id, n, 31)
    R.rn_anneal_screened(ctx, mid, R.schedule(2.0, 0.98), 40, K=32, top=2, eps=0.1)
    st = R.rn_get_chain_state(ctx, p.id, n)
    assert st["step"] == 40
    np.testing.assert_array_equal(R.rn_evaluate(ctx, p.id, st["x_cur"]), st["d_cur"])
    np.testing.assert_array_equal(R.rn_evaluate(ctx, p.id, st["x_best"]), st["d_best"])
    assert np.all(st["d_best"] <= st["d_cur"])
    for c in (0, 77, 199):
        assert O.check_params(p.net, st["x_cur"][c]) == 0
    assert np.all(st["counters"][:, 0] + st["counters"][:, 2] <= 40)
    assert np.all(st["counters"][:, 1] <= st["counters"][:, 0])


def test_screened_block_path_eps1_is_plain_annealing(ctx):
    """Block-path network (700 nodes, a block of threads per chain) with a
    width-1024 screen: with eps = 1 the screened step simulates only the plain
    proposal, so the chains are bit-identical to rn_anneal's."""
    w = synth.random_network(71, 700, lam=4.0, cap=16, n_cond=3, n_times=6, obs_frac=0.3)
    n, sweeps = 64, 12
    sched = R.schedule(5.0, 0.97)
    p = Problem(w, ctx)
    mid, D, _ = _screen(ctx, p, 1024, 1024, 5)
    R.rn_init_chains(ctx, p.id, n, 19)
    R.rn_anneal_screened(ctx, mid, sched, 5, K=32, top=2, eps=1.0)
    R.rn_anneal_screened(ctx, mid, sched, sweeps - 5, K=32, top=2, eps=1.0)
    st = R.rn_get_chain_state(ctx, p.id, n)
    ctx2 = R.rn_create(0)
    try:
        p2 = Problem(w, ctx2)
        R.rn_init_chains(ctx2, p2.id, n, 19)
        R.rn_anneal(ctx2, sched, sweeps)
        ref = R.rn_get_chain_state(ctx2, p2.id, n)
    finally:
        R.rn_destroy(ctx2)
    for k in ("x_cur", "d_cur", "x_best", "d_best", "counters"):
        np.testing.assert_array_equal(st[k], ref[k], err_msg=k)


def test_screened_block_path_step_selection(ctx):
    """One greedy screened step on a block-path network with a width-1024
    screen (its A1 from the one-hot GEMM, P x width above the per-chain
    threshold): a moved chain took a move that can be among the top 2 predicted
    (oracle prediction +- the derived bound) with exact dE <= 0; a chain that
    stayed had no candidate surely among them with dE <= 0."""
    w = synth.random_network(72, 600, lam=3.0, cap=12, n_cond=2, n_times=5, obs_frac=0.4)
    p = Problem(w, ctx)
    assert p.net.P * 1024 > (1 << 22)
    mid, D, params = _screen(ctx, p, 1024, 1024, 6)
    n, K, seed, g, top = 16, 32, 29, 0, 2
    R.rn_init_chains(ctx, p.id, n, seed)
    st0 = R.rn_get_chain_state(ctx, p.id, n)
    R.rn_anneal_screened(ctx, mid, R.schedule(1e-9, 1.0), 1, K=K, top=top, eps=0.0)
    st1 = R.rn_get_chain_state(ctx, p.id, n)
    q = gpu_view(params)
    moved = 0
    for c in range(n):
        x0 = st0["x_cur"][c]
        d0 = int(st0["d_cur"][c])
        moves = [m for m in dict.fromkeys(_candidates(p.net, x0, seed, c, g, K)) if m]
        V = np.array([np.where(np.arange(p.net.P) == j, v, x0).astype(np.int8) for j, v in moves])
        yp = O.mlp(p.net, V, q)
        b = forward_bound(p.net, V, q)
        dE = np.array([O.objective(p.net, p.tc, xv) for xv in V]) - d0
        lo, hi = yp - b, yp + b
        surely_beats = lo[None, :] > hi[:, None]
        may_beat = lo[:, None] <= hi[None, :]
        np.fill_diagonal(may_beat, False)
        possible = surely_beats.sum(axis=0) < top
        sure = may_beat.sum(axis=0) < top
        x1 = st1["x_cur"][c]
        diff = np.flatnonzero(x1 != x0)
        assert len(diff) <= 1
        if len(diff) == 1:
            moved += 1
            k = moves.index((int(diff[0]), int(x1[diff[0]])))
            assert possible[k] and dE[k] <= 0
            assert st1["d_cur"][c] == d0 + dE[k]
        else:
            assert not np.any(sure & (dE <= 0)), f"chain {c}"
            assert st1["d_cur"][c] == d0
    assert moved >= n // 4


def test_screened_block_path_invariants(ctx):
    """eps = 0.1 run on a block-path network: stored scores are exact, x_best
    holds delta_best, the constraints hold, the counters add up."""
    w = synth.random_network(73, 650, lam=4.0, cap=16, n_cond=2, n_times=6, obs_frac=0.3)
    p = Problem(w, ctx)
    mid, D, _ = _screen(ctx, p, 512, 512, 9)
    n = 48
    R.rn_init_chains(ctx, p.id, n, 37)
    R.rn_anneal_screened(ctx, mid, R.schedule(2.0, 0.98), 10, K=32, top=2, eps=0.1)
    st = R.rn_get_chain_state(ctx, p.id, n)
    assert st["step"] == 10
    np.testing.assert_array_equal(R.rn_evaluate(ctx, p.id, st["x_cur"]), st["d_cur"])
    np.testing.assert_array_equal(R.rn_evaluate(ctx, p.id, st["x_best"]), st["d_best"])
    assert np.all(st["d_best"] <= st["d_cur"])
    for c in (0, 20, 47):
        assert O.check_params(p.net, st["x_cur"][c]) == 0
    assert np.all(st["counters"][:, 0] + st["counters"][:, 2] <= 10)
    assert (st["counters"][:, 0] > 0).any()


def test_trained_screen_beats_plain_at_equal_exact_evaluations(ctx):
    """What the learned screen gains: from the same mid-anneal state, 40
    screened steps (2 exact simulations each) against 80 plain steps (1 each):
    the screened chains end with the lower mean best score."""
    w = synth.make("mtb_63n_178e")
    p = Problem(w, ctx)
    mid, D = R.rn_mlp_create(ctx, p.id, 512, 512, 1 << 18)
    params = init_weights(D, 512, 512, p.net.P, 14)
    params["W1"] *= 0.5
    R.rn_mlp_set_weights(ctx, mid, params)
    n = 1024
    sched = _logged_pairs(ctx, p, mid, n, 100, 2, 41)
    R.rn_mlp_train(ctx, mid, 400, batch=2048, lr=1e-3, seed=1)
    st0 = R.rn_get_chain_state(ctx, p.id, n)
    R.rn_anneal_screened(ctx, mid, sched, 40, K=32, top=2, eps=0.0)
    scr = R.rn_get_chain_state(ctx, p.id, n)
    R.rn_set_chain_state(ctx, p.id, 41, st0)
    R.rn_anneal(ctx, sched, 80)
    plain = R.rn_get_chain_state(ctx, p.id, n)
    m0, ms, mp = st0["d_best"].mean(), scr["d_best"].mean(), plain["d_best"].mean()
    print(f"mean best score: start {m0:.2f}, screened {ms:.2f}, plain {mp:.2f}")
    assert ms < mp
