"""Pins of the oracle's FP64 screening MLP (CPU only): a hand-computed example
and central finite differences of the loss."""
import numpy as np

from oracle import oracle as O
from paper_2506_19866_gb300 import synth
from tests.helpers import load_golden


def test_hand_computed_mlp():
    g = load_golden("mlp.json")
    net = O.Network([0, 1], [1, 0], np.zeros(2, np.uint8))
    off = O.onehot_offsets(net)
    D = int(off[-1])
    assert D == 38
    W1 = np.zeros((D, g["H1"]))
    for r, row in g["W1_rows"].items():
        W1[int(r)] = row
    params = dict(W1=W1, b1=g["b1"], W2=g["W2"], b2=g["b2"], w3=g["w3"], b3=g["b3"])
    x = np.array(g["x"], np.int8)
    # the positions the one-hot encoding sets
    pos = [int(off[j]) + list(O.domain(net, j)).index(int(x[j])) for j in range(net.P)]
    assert pos == g["active_positions"]
    y, loss, gr = O.mlp(net, x, params, target=[g["target"]])
    assert abs(y[0] - g["y"]) < 1e-12 and abs(loss - g["loss"]) < 1e-12
    assert abs(gr["b3"] - g["gb3"]) < 1e-12
    np.testing.assert_allclose(gr["w3"], g["gw3"], atol=1e-12)
    np.testing.assert_allclose(gr["b2"], g["gb2"], atol=1e-12)
    np.testing.assert_allclose(gr["W2"], g["gW2"], atol=1e-12)
    np.testing.assert_allclose(gr["b1"], g["gb1"], atol=1e-12)
    for r in range(D):
        expect = g["gW1_active_row"] if r in pos else [0.0, 0.0]
        np.testing.assert_allclose(gr["W1"][r], expect, atol=1e-12)


def test_mlp_gradients_match_finite_differences():
    w = synth.tiny(4, n_nodes=4, indeg=2)
    net = O.Network(w.src, w.dst, w.fast)
    D = int(O.onehot_offsets(net)[-1])
    rng = np.random.default_rng(0)
    H1, H2 = 6, 5
    params = dict(W1=rng.normal(0, 0.3, (D, H1)), b1=rng.normal(0, 0.3, H1),
                  W2=rng.normal(0, 0.5, (H1, H2)), b2=rng.normal(0, 0.3, H2),
                  w3=rng.normal(0, 0.5, H2), b3=0.3)
    X = O.init_chains(net, 9, 7)
    t = rng.normal(0, 1, 7)
    _, _, grads = O.mlp(net, X, params, target=t)
    eps = 1e-6
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):
        p0 = params[name]
        shape = np.shape(p0)
        flat = np.array(p0, dtype=np.float64).reshape(-1)
        for k in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            def loss_at(v):
                q = flat.copy()
                q[k] = v
                pp = dict(params)
                pp[name] = q.reshape(shape) if shape else float(q[0])
                return O.mlp(net, X, pp, target=t)[1]
            num = (loss_at(flat[k] + eps) - loss_at(flat[k] - eps)) / (2 * eps)
            ana = np.reshape(grads[name], -1)[k] if shape else grads[name]
            assert abs(num - ana) <= 1e-6 * max(1.0, abs(num)), (name, k, num, ana)


def test_bf16_rounding_pins():
    # BF16 keeps 8 significant bits: spacing 2^-7 on [1, 2); ties go to the
    # even neighbour
    from tests.mlp_util import bf16
    x = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20, 3.0,
                  -(1 + 3 * 2.0 ** -8), 2.0 ** -130], np.float32)
    want = np.array([1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, 3.0, -(1 + 2.0 ** -6), 0.0], np.float32)
    np.testing.assert_array_equal(bf16(x)[:5], want[:5])
    # subnormal input keeps its top bits (2^-130 is exact in BF16)
    assert bf16(x)[5] == np.float32(2.0 ** -130)
