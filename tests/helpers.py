"""Shared test helpers: build oracle objects from fixtures and workloads."""
import json
import os

import numpy as np

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def case_network(case):
    e = np.array(case["edges"], dtype=np.int64).reshape(-1, 5)
    net = O.Network(e[:, 0], e[:, 1], np.zeros(case["n_nodes"], np.uint8))
    x = np.concatenate([e[:, 2], e[:, 3], e[:, 4], case["u"], case["m"], case["d"]]).astype(np.int8)
    return net, x


def oracle_problem(w, noise=True):
    """Oracle network + timecourse for a synthetic workload: planted x* from the
    sampler (planted_seed, chain 0), R = its trajectories, then the noise flips."""
    from paper_2506_19866_gb300 import synth
    net = O.Network(w.src, w.dst, w.fast)
    xs = O.init_chain(net, w.planted_seed, 0)
    blank = O.Timecourse(w.init, np.zeros((w.C, w.T, w.N), np.uint8), w.observed, w.knockout)
    _, traj = O.objective(net, blank, xs, return_traj=True)
    flipped = np.zeros(traj.shape, dtype=bool)
    R = traj
    if noise and w.noise_frac > 0:
        R, flipped = synth.flip_noise(traj, w.observed, w.noise_frac, w.noise_seed)
    tc = O.Timecourse(w.init, R, w.observed, w.knockout)
    return net, tc, xs, flipped
