"""Seeded synthetic workloads shaped like the paper's two systems and like the
benchmark configurations.

This module holds none of the method's arithmetic.  It draws topologies
(random signed digraphs are signed only later, by the parameters), speed
classes, experimental conditions, observation masks and noise flips with
numpy's PCG64, from fixed seeds.  The planted parameter vector and the
reference data R are produced by whoever simulates: the oracle in the tests,
the CUDA library in the benchmark (both from the same seeds; the tests check
that the two agree).

Input recipe (the paper's shapes, Section 2.5): about one third of the nodes
fast (u in {10,11,12}); each condition is an initial state drawn uniformly
from {0,1,2}^N, condition 0 without knockout and every other condition with
one random node knocked out; observation masks are Bernoulli per entry (or a
node subset over all time points for the paper-shaped presets); noise flips a
fraction of the observed entries to a different value.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    src: np.ndarray            # [E] int32
    dst: np.ndarray            # [E] int32
    fast: np.ndarray           # [N] uint8
    init: np.ndarray           # [C][N] uint8
    knockout: np.ndarray       # [C][N] uint8
    observed: np.ndarray       # [C][T][N] uint8
    n_times: int
    planted_seed: int          # x* = sampler(planted_seed, chain 0)
    noise_frac: float
    noise_seed: int
    chain_seed: int            # Philox key of the annealing chains
    n_chains: int
    sweeps: int
    T0: float
    alpha: float
    extra: dict = field(default_factory=dict)

    @property
    def N(self):
        return int(self.fast.shape[0])

    @property
    def E(self):
        return int(self.src.shape[0])

    @property
    def P(self):
        return 3 * self.E + 3 * self.N

    @property
    def C(self):
        return int(self.init.shape[0])

    @property
    def T(self):
        return int(self.n_times)


def _canonical(src, dst):
    order = np.lexsort((src, dst))
    return src[order].astype(np.int32), dst[order].astype(np.int32)


def _ensure_out_edges(src, dst, n_nodes, rng):
    """Rewire edges so that every node has at least one out-edge, keeping every
    node's in-degree: an edge a -> b whose source has out-degree >= 2 is
    re-pointed to come from the node that has none."""
    src = src.copy()
    for _ in range(8 * n_nodes):
        outdeg = np.bincount(src, minlength=n_nodes)
        lonely = np.flatnonzero(outdeg == 0)
        if lonely.size == 0:
            return src
        i = int(lonely[0])
        existing = set(zip(src.tolist(), dst.tolist()))
        cand = [e for e in range(src.size)
                if outdeg[src[e]] >= 2 and dst[e] != i and (i, int(dst[e])) not in existing]
        if not cand:
            raise ValueError("cannot give every node an out-edge")
        e = cand[int(rng.integers(len(cand)))]
        src[e] = i
    raise ValueError("out-edge repair did not converge")


def random_digraph(n_nodes, indegrees, rng):
    """Each node i draws indegrees[i] distinct sources among the other nodes;
    then sources are rewired so that every node also has an out-edge."""
    src, dst = [], []
    for i in range(n_nodes):
        others = np.array([j for j in range(n_nodes) if j != i])
        k = int(min(indegrees[i], others.size))
        for j in rng.choice(others, size=k, replace=False):
            src.append(int(j))
            dst.append(i)
    src = np.array(src, dtype=np.int64)
    dst = np.array(dst, dtype=np.int64)
    src = _ensure_out_edges(src, dst, n_nodes, rng)
    return _canonical(src, dst)


def digraph_with_edges(n_nodes, n_edges, rng):
    """A random simple digraph with exactly n_edges edges in which every node has
    at least one in-edge and one out-edge (the paper's networks are closed-loop,
    Section 2.5.3)."""
    if n_edges < n_nodes or n_edges > n_nodes * (n_nodes - 1):
        raise ValueError("edge count out of range")
    indeg = np.ones(n_nodes, dtype=np.int64)
    for i in rng.choice(n_nodes, size=n_edges - n_nodes, replace=True):
        indeg[i] += 1
    while indeg.max() > n_nodes - 1:
        hi = int(np.argmax(indeg))
        lo = int(np.argmin(indeg))
        indeg[hi] -= 1
        indeg[lo] += 1
    return random_digraph(n_nodes, indeg, rng)


def speed_classes(n_nodes, rng, frac=1.0 / 3.0):
    fast = np.zeros(n_nodes, dtype=np.uint8)
    fast[rng.choice(n_nodes, size=int(round(frac * n_nodes)), replace=False)] = 1
    return fast


def conditions(n_nodes, n_cond, rng):
    init = rng.integers(0, 3, size=(n_cond, n_nodes)).astype(np.uint8)
    ko = np.zeros((n_cond, n_nodes), dtype=np.uint8)
    for c in range(1, n_cond):
        ko[c, int(rng.integers(n_nodes))] = 1
    return init, ko


def bernoulli_mask(n_cond, n_times, n_nodes, frac, rng):
    return (rng.random((n_cond, n_times, n_nodes)) < frac).astype(np.uint8)


def node_subset_mask(n_cond, n_times, n_nodes, n_observed, rng):
    obs = np.zeros((n_cond, n_times, n_nodes), dtype=np.uint8)
    obs[:, :, rng.choice(n_nodes, size=n_observed, replace=False)] = 1
    return obs


def flip_noise(ref, observed, frac, seed):
    """Flip round(frac * n_obs) observed entries of R to a uniformly chosen
    different value.  Returns (R_noisy, flipped_mask)."""
    rng = np.random.default_rng(seed)
    ref = np.array(ref, dtype=np.uint8, copy=True)
    idx = np.flatnonzero(observed.reshape(-1))
    n_flip = int(round(frac * idx.size))
    flipped = np.zeros(ref.size, dtype=bool)
    if n_flip:
        pick = rng.choice(idx, size=n_flip, replace=False)
        shift = rng.integers(1, 3, size=n_flip).astype(np.uint8)
        flat = ref.reshape(-1)
        flat[pick] = (flat[pick] + shift) % 3
        flipped[pick] = True
    return ref, flipped.reshape(ref.shape)


def _poisson_indegree(n_nodes, lam, cap, rng):
    return np.clip(rng.poisson(lam, size=n_nodes), 1, cap)


def plain_alpha(T0, T_end, sweeps):
    """Geometric factor that cools T0 to T_end over the given number of sweeps."""
    return math.exp(math.log(T_end / T0) / sweeps)


# Sweep-per-level cooling of the small configuration: T0 = 10, alpha = 0.995
# over 2000 sweeps ends at 10 * 0.995^2000; the larger runs span the same range.
T_END_PLAIN = 10.0 * 0.995 ** 2000


def make(name: str) -> Workload:
    """Build a named workload (deterministic)."""
    if name == "n15_c3_t11":
        rng = np.random.default_rng(1001)
        src, dst = random_digraph(15, np.full(15, 3), rng)
        fast = speed_classes(15, rng)
        init, ko = conditions(15, 3, rng)
        obs = bernoulli_mask(3, 11, 15, 0.3, np.random.default_rng(3001))
        return Workload(name, src, dst, fast, init, ko, obs, 11, planted_seed=2001,
                        noise_frac=0.0, noise_seed=4001, chain_seed=0, n_chains=64,
                        sweeps=2000, T0=10.0, alpha=0.995)
    if name == "n120_c8_t21":
        rng = np.random.default_rng(1002)
        src, dst = random_digraph(120, _poisson_indegree(120, 5.0, 10, rng), rng)
        fast = speed_classes(120, rng)
        init, ko = conditions(120, 8, rng)
        obs = bernoulli_mask(8, 21, 120, 0.2, np.random.default_rng(3002))
        return Workload(name, src, dst, fast, init, ko, obs, 21, planted_seed=2002,
                        noise_frac=0.05, noise_seed=4002, chain_seed=0, n_chains=4096,
                        sweeps=100_000, T0=10.0,
                        alpha=plain_alpha(10.0, T_END_PLAIN, 100_000))
    if name == "hpg_9n_25e":
        # Shaped like the HPG axis: 9 nodes, 25 edges (P = 102), 3 fast nodes,
        # 5 observed nodes over 20 time points, one time course.
        rng = np.random.default_rng(1101)
        src, dst = digraph_with_edges(9, 25, rng)
        fast = speed_classes(9, rng)
        init, ko = conditions(9, 1, rng)
        obs = node_subset_mask(1, 20, 9, 5, np.random.default_rng(3101))
        return Workload(name, src, dst, fast, init, ko, obs, 20, planted_seed=2101,
                        noise_frac=0.0, noise_seed=4101, chain_seed=0, n_chains=1024,
                        sweeps=2000, T0=10.0, alpha=0.995)
    if name == "mtb_63n_178e":
        # Shaped like the Mtb host-pathogen network: 63 nodes, 178 edges
        # (P = 723), one third fast, 35 observed nodes over 20 time points.
        rng = np.random.default_rng(1102)
        src, dst = digraph_with_edges(63, 178, rng)
        fast = speed_classes(63, rng)
        init, ko = conditions(63, 1, rng)
        obs = node_subset_mask(1, 20, 63, 35, np.random.default_rng(3102))
        return Workload(name, src, dst, fast, init, ko, obs, 20, planted_seed=2102,
                        noise_frac=0.0, noise_seed=4102, chain_seed=0, n_chains=4096,
                        sweeps=20_000, T0=10.0, alpha=plain_alpha(10.0, T_END_PLAIN, 20_000))
    if name == "n2000_c16_t33":
        # Scale-up network: 2000 nodes, in-degree Poisson(6) (floored at 1, capped
        # at the block path's 31, which this draw never reaches), 16 conditions,
        # 32 update steps (T = 33 points with t0), 10% of entries observed, no
        # noise; 16384 chains.
        rng = np.random.default_rng(1005)
        src, dst = random_digraph(2000, _poisson_indegree(2000, 6.0, 31, rng), rng)
        fast = speed_classes(2000, rng)
        init, ko = conditions(2000, 16, rng)
        obs = bernoulli_mask(16, 33, 2000, 0.1, np.random.default_rng(3005))
        return Workload(name, src, dst, fast, init, ko, obs, 33, planted_seed=2005,
                        noise_frac=0.0, noise_seed=4005, chain_seed=0, n_chains=16384,
                        sweeps=2000, T0=10.0, alpha=0.995)
    raise KeyError(name)


WORKLOADS = ("n15_c3_t11", "n120_c8_t21", "hpg_9n_25e", "mtb_63n_178e")
# networks above 512 nodes (a block of threads per chain)
LARGE_WORKLOADS = ("n2000_c16_t33",)


def make_batch(n_nets=256, total_chains=65536, seed=1003, n_min=10, n_max=300, max_indeg=16,
               lam=4.0, obs_frac=0.2):
    """Many independent networks of uneven size annealed together: node counts
    log-uniform in [n_min, n_max], in-degree Poisson(lam) (at least 1, at most
    max_indeg), 2-12 conditions, 8-32 update steps, obs_frac observed entries, and
    chains per network proportional to its parameter count (total_chains in
    all, at least one each).  Returns a list of Workloads."""
    rng = np.random.default_rng(seed)
    nets = []
    for b in range(n_nets):
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        cap = min(N - 1, max_indeg)
        src, dst = random_digraph(N, np.clip(rng.poisson(lam, size=N), 1, cap), rng)
        fast = speed_classes(N, rng)
        C = int(rng.integers(2, 13))
        T = int(rng.integers(8, 33)) + 1
        init, ko = conditions(N, C, rng)
        obs = bernoulli_mask(C, T, N, obs_frac, rng)
        nets.append(Workload(f"batch{b}", src, dst, fast, init, ko, obs, T,
                             planted_seed=20000 + b, noise_frac=0.0, noise_seed=30000 + b,
                             chain_seed=b, n_chains=1, sweeps=2000, T0=10.0, alpha=0.995))
    P = np.array([w.P for w in nets], dtype=np.float64)
    share = np.maximum(1, np.floor(total_chains * P / P.sum())).astype(np.int64)
    rest = total_chains - int(share.sum())
    for b in np.argsort(-P)[:max(0, rest)]:
        share[b] += 1
    for w, n in zip(nets, share):
        w.n_chains = int(n)
    return nets


def make_scaleup():
    """The scale-up set: the 2000-node, 16-condition network with its 16384
    chains, and 63 networks of 100-1000 nodes (log-uniform, in-degree
    Poisson(6), 10% observed, 2-12 conditions, 8-32 update steps) with 16384
    chains in all, proportional to their parameter counts."""
    big = make("n2000_c16_t33")
    small = make_batch(n_nets=63, total_chains=16384, seed=1006, n_min=100, n_max=1000,
                       max_indeg=24, lam=6.0, obs_frac=0.1)
    return [big] + small


def tiny(seed, n_nodes=4, indeg=2, n_cond=2, n_times=6, obs_frac=0.5):
    """A small random workload for parity and brute-force tests."""
    rng = np.random.default_rng(seed)
    src, dst = random_digraph(n_nodes, np.full(n_nodes, min(indeg, n_nodes - 1)), rng)
    fast = speed_classes(n_nodes, rng)
    init, ko = conditions(n_nodes, n_cond, rng)
    obs = bernoulli_mask(n_cond, n_times, n_nodes, obs_frac, rng)
    return Workload(f"tiny{seed}", src, dst, fast, init, ko, obs, n_times,
                    planted_seed=seed + 7, noise_frac=0.0, noise_seed=seed + 11,
                    chain_seed=seed + 13, n_chains=8, sweeps=50, T0=10.0, alpha=0.995)


def random_network(seed, n_nodes, lam, cap, n_cond, n_times, obs_frac):
    """A random workload with Poisson in-degrees (for size sweeps and tests)."""
    rng = np.random.default_rng(seed)
    src, dst = random_digraph(n_nodes, _poisson_indegree(n_nodes, lam, cap, rng), rng)
    fast = speed_classes(n_nodes, rng)
    init, ko = conditions(n_nodes, n_cond, rng)
    obs = bernoulli_mask(n_cond, n_times, n_nodes, obs_frac, rng)
    return Workload(f"rand{seed}_{n_nodes}", src, dst, fast, init, ko, obs, n_times,
                    planted_seed=seed + 7, noise_frac=0.0, noise_seed=seed + 11,
                    chain_seed=seed + 13, n_chains=64, sweeps=100, T0=10.0, alpha=0.995)
