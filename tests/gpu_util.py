"""Helpers of the GPU tests: one problem built for both the oracle and the library."""
import numpy as np

from oracle import oracle as O
from paper_2506_19866_gb300 import rnanneal as R
from tests.helpers import oracle_problem


class Problem:
    def __init__(self, w, ctx, noise=True, frozen=None, frozen_val=None, sync=False,
                 async_sel=None):
        self.w = w
        base, tc, xs, flipped = oracle_problem(w, noise=noise)
        self.xs = xs
        self.flipped = flipped
        self.net = O.Network(w.src, w.dst, w.fast, frozen, frozen_val, sync=sync,
                             async_sel=async_sel)
        self.tc = tc
        self.ctx = ctx
        self.id = R.rn_load_network(ctx, w.src, w.dst, w.fast, frozen, frozen_val)
        R.rn_load_timecourse(ctx, self.id, w.init, tc.ref, w.observed, w.knockout)
        if sync:
            R.rn_set_update_scheme(ctx, self.id, 1)
        if async_sel is not None:
            R.rn_set_update_scheme(ctx, self.id, 2, async_sel)

    @property
    def shape(self):
        return (self.w.C, self.w.T, self.w.N)


def random_vectors(net, n, seed):
    """Vectors drawn uniformly from the domains (constraints not enforced)."""
    rng = np.random.default_rng(seed)
    X = np.zeros((n, net.P), np.int8)
    for j in range(net.P):
        dom = O.domain(net, j)
        X[:, j] = dom[rng.integers(len(dom), size=n)]
    return X
