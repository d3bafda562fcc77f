"""The seeded synthetic inputs follow their stated recipe (no GPU): the
paper-shaped presets have the paper's parameter counts (Sections 2.5 and 3),
the benchmark workloads have the sizes the benchmark reports, every network is
a simple digraph in canonical edge order with an in- and an out-edge per node,
and the generators are deterministic."""
import numpy as np
import pytest

from paper_2506_19866_gb300 import synth

ALL = synth.WORKLOADS + synth.LARGE_WORKLOADS


def _structure(w):
    src, dst = np.asarray(w.src), np.asarray(w.dst)
    assert (src != dst).all()                                   # no self-loops
    pairs = list(zip(dst.tolist(), src.tolist()))
    assert pairs == sorted(set(pairs))                          # sorted by (dst, src), no duplicates
    assert (np.bincount(dst, minlength=w.N) >= 1).all()
    assert (np.bincount(src, minlength=w.N) >= 1).all()
    assert int(w.fast.sum()) == round(w.N / 3)                  # one third fast
    assert set(np.unique(w.init)) <= {0, 1, 2}
    assert w.knockout[0].sum() == 0                             # condition 0: no knockout
    assert (w.knockout[1:].sum(axis=1) == 1).all()              # the others: one node each
    assert w.observed.shape == (w.C, w.T, w.N)


@pytest.mark.parametrize("name", ALL)
def test_workload_structure_and_determinism(name):
    w = synth.make(name)
    _structure(w)
    v = synth.make(name)
    for k in ("src", "dst", "fast", "init", "knockout", "observed"):
        np.testing.assert_array_equal(getattr(w, k), getattr(v, k))


@pytest.mark.parametrize("name,N,E,P,C,T,chains,n_obs", [
    ("hpg_9n_25e", 9, 25, 102, 1, 20, 1024, 100),       # P = 102 as Section 3 prints
    ("mtb_63n_178e", 63, 178, 723, 1, 20, 4096, 700),   # P = 723 as Section 3 prints
    ("n15_c3_t11", 15, 45, 180, 3, 11, 64, None),
    ("n120_c8_t21", 120, 581, 2103, 8, 21, 4096, None),
    ("n2000_c16_t33", 2000, 12113, 42339, 16, 33, 16384, None),
])
def test_workload_sizes(name, N, E, P, C, T, chains, n_obs):
    w = synth.make(name)
    assert (w.N, w.E, w.P, w.C, w.T, w.n_chains) == (N, E, P, C, T, chains)
    if n_obs is not None:
        # a node subset observed at every time point
        assert int(w.observed.sum()) == n_obs
        rows = w.observed.reshape(-1, w.N)
        assert (rows == rows[0]).all()


def test_presets_in_degrees_and_observation_rates():
    w = synth.make("n15_c3_t11")
    assert (np.bincount(w.dst, minlength=w.N) == 3).all()
    for name, frac in (("n15_c3_t11", 0.3), ("n120_c8_t21", 0.2), ("n2000_c16_t33", 0.1)):
        w = synth.make(name)
        n = w.observed.size
        assert abs(w.observed.sum() / n - frac) < 4 * np.sqrt(frac * (1 - frac) / n)
    deg = np.bincount(synth.make("n120_c8_t21").dst, minlength=120)
    assert deg.min() >= 1 and deg.max() <= 10


def test_batch256_recipe():
    nets = synth.make_batch()
    assert len(nets) == 256 and sum(w.n_chains for w in nets) == 65536
    assert sum(w.E for w in nets) == 86938 and sum(w.P for w in nets) == 325752
    assert int(np.median([w.N for w in nets])) == 59
    for w in nets:
        _structure(w)
        assert 10 <= w.N <= 300 and 2 <= w.C <= 12 and 9 <= w.T <= 33 and w.n_chains >= 1
        assert np.bincount(w.dst, minlength=w.N).max() <= 16
    # chains in proportion to the parameter count (within the integer split)
    P = np.array([w.P for w in nets], float)
    share = np.array([w.n_chains for w in nets])
    assert np.abs(share - 65536 * P / P.sum()).max() < 2


def test_scaleup_recipe():
    nets = synth.make_scaleup()
    assert len(nets) == 64 and nets[0].name == "n2000_c16_t33"
    assert sum(w.n_chains for w in nets) == 32768 and sum(w.n_chains for w in nets[1:]) == 16384
    assert sum(w.P for w in nets) == 553293
    for w in nets[1:]:
        _structure(w)
        assert 100 <= w.N <= 1000 and np.bincount(w.dst, minlength=w.N).max() <= 24
