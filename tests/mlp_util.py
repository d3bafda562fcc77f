"""Helpers of the surrogate tests: BF16 rounding, seeded weights, and the
forward-error bound of the GPU's mixed-precision MLP against the FP64 oracle.

The GPU computes y = b3 + w3 . relu(b2 + W2^T q(relu(b1 + W1^T onehot(x))))
with W1, W2 rounded to BF16 (the oracle is given the same rounded weights),
the hidden vector h1 rounded to BF16 (q), and every sum accumulated in FP32.
Rounding to nearest has relative error at most u = 2^-8 for BF16 (8
significant bits).  A sum of n terms accumulated in FP32 is off by at most
gamma(n) = n e / (1 - n e) times the sum of the terms' magnitudes, whatever
the order (Higham, Accuracy and Stability of Numerical Algorithms, 2nd ed.,
Sec. 3.1), with e = 2^-24 for round-to-nearest; e = 2^-22 is taken here, which
also covers accumulators that truncate instead of rounding.  BF16 x BF16
products are exact in FP32.  ReLU is 1-Lipschitz.  So, per vector:
    |da1| <= gamma(P + 1) (|b1| + sum_j |W1[row_j]|)
    |dh1| <= |da1| + u (h1 + |da1|)                       (q and FP32)
    |da2| <= |W2|^T |dh1| + gamma(H1 + 1) (|W2|^T (h1 + |dh1|) + |b2|)
    |dy|  <= |w3| . |da2| + gamma(H2 + 2) (|w3| . (h2 + |da2|) + |b3|)
with h1, h2 the exact (oracle) activations.

That worst case adds every rounding error with the same sign.  To first
order (ReLU masks fixed) the output error is linear in the element errors:
    dy = sum_h c_h e_h + sum_k w3_k [a2_k > 0] f_k + z,
    c_h = sum_k w3_k [a2_k > 0] W2_hk,
with e_h the error of the BF16 h1 entry (|e_h| <= ulp(h1_h) / 2 + the FP32
layer-1 bound), f_k the FP32 error of a2_k (gamma(H1 + 1) times its terms'
magnitudes) and z the FP32 error of the final dot product.  Treating element
errors as independent and zero-mean (the model of Higham & Mary, "A new
approach to probabilistic rounding error analysis", SIAM J. Sci. Comput. 41,
2019), Hoeffding's inequality bounds a sum of independent X_i with
|X_i| <= b_i by lambda sqrt(sum b_i^2) except with probability
2 exp(-lambda^2 / 2).  The same model bounds one FP32 sum of n terms by
lambda sqrt(n) e times its terms' magnitudes (ibid., Theorem 2.4).
stat_tolerance() takes lambda = 6 throughout, and the worst case for z.
"""
import numpy as np

from oracle import oracle as O

U_BF16 = 2.0 ** -8


def bf16(a):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def gamma(n):
    e = n * 2.0 ** -22
    return e / (1.0 - e)


def gamma_prob(n, lam=6.0):
    return lam * np.sqrt(n) * 2.0 ** -22


def init_weights(D, H1, H2, P, seed):
    """Seeded weights with O(1) activations: each layer-1 unit sums P rows."""
    rng = np.random.default_rng(seed)
    return dict(W1=(rng.standard_normal((D, H1)) / np.sqrt(P)).astype(np.float32),
                b1=(0.1 * rng.standard_normal(H1)).astype(np.float32),
                W2=(rng.standard_normal((H1, H2)) * np.sqrt(2.0 / H1)).astype(np.float32),
                b2=(0.1 * rng.standard_normal(H2)).astype(np.float32),
                w3=(rng.standard_normal(H2) / np.sqrt(H2)).astype(np.float32),
                b3=float(rng.standard_normal() * 0.1))


def gpu_view(params):
    """The weights the GPU multiplies with: W1 and W2 rounded to BF16."""
    q = dict(params)
    q["W1"] = bf16(params["W1"])
    q["W2"] = bf16(params["W2"])
    return q


def onehot(net, X):
    off = O.onehot_offsets(net)
    D = int(off[-1])
    OH = np.zeros((X.shape[0], D))
    for j in range(net.P):
        dom = O.domain(net, j)
        pos = np.searchsorted(dom, X[:, j])
        OH[np.arange(X.shape[0]), off[j] + pos] = 1.0
    return OH


def bf16_ulp(h):
    """Spacing of BF16 numbers at |h| (8 significant bits); 0 where h = 0."""
    h = np.abs(np.asarray(h, np.float64))
    e = np.floor(np.log2(np.where(h > 0, h, 1.0)))
    return np.where(h > 0, 2.0 ** (e - 7), 0.0)


def stat_tolerance(net, X, q, lam=6.0):
    """Per-vector probabilistic tolerance of |y_gpu - y_oracle| (the module docstring)."""
    OH = onehot(net, X)
    W1, b1, W2, b2, w3 = (np.asarray(q[k], np.float64) for k in ("W1", "b1", "W2", "b2", "w3"))
    b3 = float(q["b3"])
    P, H1, H2 = net.P, W1.shape[1], W2.shape[1]
    a1 = b1 + OH @ W1
    h1 = np.maximum(a1, 0)
    a2 = b2 + h1 @ W2
    h2 = np.maximum(a2, 0)
    act = (a2 > 0) * w3                               # [n][H2]
    c = act @ W2.T                                    # [n][H1]
    e = bf16_ulp(h1) / 2 + gamma_prob(P + 1, lam) * (np.abs(b1) + OH @ np.abs(W1))
    f = gamma_prob(H1 + 1, lam) * ((h1 + e) @ np.abs(W2) + np.abs(b2))
    z = gamma(H2 + 2) * ((h2 + f) @ np.abs(w3) + abs(b3))
    return lam * np.sqrt(np.sum((c * e) ** 2, axis=1)) + \
        lam * np.sqrt(np.sum((act * f) ** 2, axis=1)) + z


def forward_bound(net, X, q):
    """Per-vector worst-case bound on |y_gpu - y_oracle| for weights q (already
    BF16-rounded)."""
    OH = onehot(net, X)
    W1, b1, W2, b2, w3 = (np.asarray(q[k], np.float64) for k in ("W1", "b1", "W2", "b2", "w3"))
    b3 = float(q["b3"])
    P, H1, H2 = net.P, W1.shape[1], W2.shape[1]
    a1 = b1 + OH @ W1
    h1 = np.maximum(a1, 0)
    da1 = gamma(P + 1) * (np.abs(b1) + OH @ np.abs(W1))
    dh1 = da1 + U_BF16 * (h1 + da1)
    h2 = np.maximum(b2 + h1 @ W2, 0)
    da2 = dh1 @ np.abs(W2) + gamma(H1 + 1) * ((h1 + dh1) @ np.abs(W2) + np.abs(b2))
    return np.abs(w3) @ da2.T + gamma(H2 + 2) * ((h2 + da2) @ np.abs(w3) + abs(b3))


def spearman(a, b):
    """Rank correlation (average ranks on ties)."""
    from scipy.stats import spearmanr
    return float(spearmanr(a, b).correlation)
