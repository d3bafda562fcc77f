"""ctypes wrapper around the plain CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library under
paper_2506_19866_gb300/.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ORC_OK, ORC_EINVAL, ORC_ECONSTRAINT, ORC_ENOMEM = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain C, -O2, no vector intrinsics).
    ORC_LIB names a prebuilt library to load instead: the pin tests run against
    oracle builds with a planted mistake that way (tests/test_oracle_mutants.py)."""
    if os.environ.get("ORC_LIB"):
        return os.environ["ORC_LIB"]
    stale =(not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h")))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Net(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("fast", ctypes.c_void_p), ("frozen", ctypes.c_void_p),
                ("frozen_val", ctypes.c_void_p), ("sync", ctypes.c_int32),
                ("n_cond_sel", ctypes.c_int32), ("n_times_sel", ctypes.c_int32),
                ("async_sel", ctypes.c_void_p)]


class _TC(ctypes.Structure):
    _fields_ = [("n_cond", ctypes.c_int32), ("n_times", ctypes.c_int32),
                ("init", ctypes.c_void_p), ("knockout", ctypes.c_void_p),
                ("ref", ctypes.c_void_p), ("observed", ctypes.c_void_p)]


class _Sched(ctypes.Structure):
    _fields_ = [("T0", ctypes.c_double), ("alpha", ctypes.c_double),
                ("iters_per_level", ctypes.c_int64), ("reset_to_best", ctypes.c_int32),
                ("global_sync", ctypes.c_int32), ("sync_group", ctypes.c_int32)]


class _Chains(ctypes.Structure):
    _fields_ = [("x_cur", ctypes.c_void_p), ("x_best", ctypes.c_void_p),
                ("d_cur", ctypes.c_void_p), ("d_best", ctypes.c_void_p),
                ("n_accept", ctypes.c_void_p), ("n_uphill", ctypes.c_void_p),
                ("n_null", ctypes.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        sig = {
            "orc_n_params": (ctypes.c_int32, [P(_Net)]),
            "orc_domain": (ctypes.c_int32, [P(_Net), ctypes.c_int32, ctypes.c_void_p]),
            "orc_philox4x32_10": (None, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                         ctypes.c_void_p]),
            "orc_threshold": (ctypes.c_uint32, [ctypes.c_double, ctypes.c_int64]),
            "orc_level_temperature": (ctypes.c_double, [ctypes.c_double, ctypes.c_double,
                                                        ctypes.c_int64]),
            "orc_count_levels": (ctypes.c_int32, [ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double]),
            "orc_weights": (None, [P(_Net), P(_TC), ctypes.c_void_p]),
            "orc_simulate": (ctypes.c_int32, [P(_Net), P(_TC), ctypes.c_void_p, ctypes.c_int32,
                                              ctypes.c_void_p]),
            "orc_score_trajectory": (ctypes.c_int32, [P(_Net), P(_TC), ctypes.c_void_p]),
            "orc_objective": (ctypes.c_int32, [P(_Net), P(_TC), ctypes.c_void_p,
                                               ctypes.c_void_p]),
            "orc_check_params": (ctypes.c_int32, [P(_Net), ctypes.c_void_p]),
            "orc_propose": (ctypes.c_int32, [P(_Net), ctypes.c_void_p, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
            "orc_init_chain": (ctypes.c_int32, [P(_Net), ctypes.c_uint64, ctypes.c_int32,
                                                ctypes.c_void_p]),
            "orc_anneal": (ctypes.c_int32, [P(_Net), P(_TC), P(_Sched), ctypes.c_uint64,
                                            ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_int64, P(_Chains)]),
            "orc_bruteforce": (ctypes.c_int64, [P(_Net), P(_TC), ctypes.c_void_p,
                                                ctypes.c_void_p]),
            "orc_onehot_offsets": (ctypes.c_int32, [P(_Net), ctypes.c_void_p]),
            "orc_mlp": (ctypes.c_int32, [P(_Net), ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
                        + [ctypes.c_void_p] * 5 + [ctypes.c_double]
                        + [ctypes.c_void_p] * 8),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Network:
    """Topology + speed classes (+ optional fixed parameters) as the oracle sees them."""

    def __init__(self, src, dst, fast, frozen=None, frozen_val=None, sync=False, async_sel=None):
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.dst = np.ascontiguousarray(dst, dtype=np.int32)
        self.fast = np.ascontiguousarray(fast, dtype=np.uint8)
        self.N = int(self.fast.shape[0])
        self.E = int(self.src.shape[0])
        self.P = 3 * self.E + 3 * self.N
        self.frozen = None if frozen is None else np.ascontiguousarray(frozen, dtype=np.uint8)
        self.frozen_val = (None if frozen_val is None
                           else np.ascontiguousarray(frozen_val, dtype=np.int8))
        self.sync = bool(sync)
        # asynchronous scheme: [C][T] node selected at each step (-1: none)
        self.async_sel = (None if async_sel is None
                          else np.ascontiguousarray(async_sel, dtype=np.int32))
        C_sel, T_sel = (0, 0) if self.async_sel is None else self.async_sel.shape
        self.s = _Net(self.N, self.E, _ptr(self.src), _ptr(self.dst), _ptr(self.fast),
                      _ptr(self.frozen), _ptr(self.frozen_val), int(self.sync), C_sel, T_sel,
                      _ptr(self.async_sel))


class Timecourse:
    """Conditions, reference data R and observation mask."""

    def __init__(self, init, ref, observed, knockout=None):
        self.init = np.ascontiguousarray(init, dtype=np.uint8)
        self.ref = np.ascontiguousarray(ref, dtype=np.uint8)
        self.observed = np.ascontiguousarray(observed, dtype=np.uint8)
        self.knockout = None if knockout is None else np.ascontiguousarray(knockout, dtype=np.uint8)
        self.C, self.T = int(self.ref.shape[0]), int(self.ref.shape[1])
        self.s = _TC(self.C, self.T, _ptr(self.init), _ptr(self.knockout), _ptr(self.ref),
                     _ptr(self.observed))


def n_params(net):
    return lib().orc_n_params(ctypes.byref(net.s))


def domain(net, j):
    vals = np.zeros(6, dtype=np.int8)
    n = lib().orc_domain(ctypes.byref(net.s), int(j), vals.ctypes.data)
    return vals[:n].copy()


def philox(seed, ctr):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF, c.ctypes.data,
                            out.ctypes.data)
    return out


def threshold(T, dE):
    return int(lib().orc_threshold(float(T), int(dE)))


def level_temperature(T0, alpha, level):
    return float(lib().orc_level_temperature(float(T0), float(alpha), int(level)))


def count_levels(T, T_min, rho):
    return int(lib().orc_count_levels(float(T), float(T_min), float(rho)))


def weights(net, tc):
    W = np.zeros((tc.C, tc.T, net.N), dtype=np.uint8)
    lib().orc_weights(ctypes.byref(net.s), ctypes.byref(tc.s), W.ctypes.data)
    return W


def simulate(net, tc, x, c):
    x = np.ascontiguousarray(x, dtype=np.int8)
    S = np.zeros((tc.T, net.N), dtype=np.uint8)
    rc = lib().orc_simulate(ctypes.byref(net.s), ctypes.byref(tc.s), x.ctypes.data, int(c),
                            S.ctypes.data)
    if rc != ORC_OK:
        raise RuntimeError(f"orc_simulate: {rc}")
    return S


def score_trajectory(net, tc, traj):
    traj = np.ascontiguousarray(traj, dtype=np.uint8)
    return int(lib().orc_score_trajectory(ctypes.byref(net.s), ctypes.byref(tc.s),
                                          traj.ctypes.data))


def objective(net, tc, x, return_traj=False):
    x = np.ascontiguousarray(x, dtype=np.int8)
    traj = np.zeros((tc.C, tc.T, net.N), dtype=np.uint8) if return_traj else None
    y = lib().orc_objective(ctypes.byref(net.s), ctypes.byref(tc.s), x.ctypes.data,
                            _ptr(traj))
    if y < 0:
        raise RuntimeError(f"orc_objective: {y}")
    return (int(y), traj) if return_traj else int(y)


def check_params(net, x):
    x = np.ascontiguousarray(x, dtype=np.int8)
    return int(lib().orc_check_params(ctypes.byref(net.s), x.ctypes.data))


def propose(net, x, r0, r1):
    """Returns (moved, j, v): moved is False for a null move."""
    x = np.ascontiguousarray(x, dtype=np.int8)
    j = ctypes.c_int32(-1)
    v = ctypes.c_int8(0)
    moved = lib().orc_propose(ctypes.byref(net.s), x.ctypes.data, int(r0) & 0xFFFFFFFF,
                              int(r1) & 0xFFFFFFFF, ctypes.addressof(j), ctypes.addressof(v))
    return bool(moved), int(j.value), int(v.value)


def init_chain(net, seed, chain):
    x = np.zeros(net.P, dtype=np.int8)
    rc = lib().orc_init_chain(ctypes.byref(net.s), int(seed), int(chain), x.ctypes.data)
    if rc != ORC_OK:
        raise ValueError(f"orc_init_chain: {rc}")
    return x


def init_chains(net, seed, n_chains, chain_ids=None):
    ids = range(n_chains) if chain_ids is None else chain_ids
    return np.stack([init_chain(net, seed, c) for c in ids]) if len(ids) else \
        np.zeros((0, net.P), dtype=np.int8)


class Schedule:
    def __init__(self, T0, alpha, iters_per_level=1, reset_to_best=False, global_sync=False,
                 sync_group=0):
        self.T0, self.alpha = float(T0), float(alpha)
        self.iters_per_level = int(iters_per_level)
        self.reset_to_best, self.global_sync = bool(reset_to_best), bool(global_sync)
        self.sync_group = int(sync_group)
        self.s = _Sched(self.T0, self.alpha, self.iters_per_level, int(self.reset_to_best),
                        int(self.global_sync), self.sync_group)


class Chains:
    """Per-chain annealing state (x_cur, x_best, objectives, counters)."""

    def __init__(self, x_cur, d_cur, x_best=None, d_best=None, n_accept=None, n_uphill=None,
                 n_null=None):
        n = x_cur.shape[0]
        self.x_cur = np.ascontiguousarray(x_cur, dtype=np.int8).copy()
        self.x_best = (self.x_cur.copy() if x_best is None
                       else np.ascontiguousarray(x_best, dtype=np.int8).copy())
        self.d_cur = np.ascontiguousarray(d_cur, dtype=np.int32).copy()
        self.d_best = (self.d_cur.copy() if d_best is None
                       else np.ascontiguousarray(d_best, dtype=np.int32).copy())
        z = np.zeros(n, dtype=np.int64)
        self.n_accept = z.copy() if n_accept is None else np.asarray(n_accept, np.int64).copy()
        self.n_uphill = z.copy() if n_uphill is None else np.asarray(n_uphill, np.int64).copy()
        self.n_null = z.copy() if n_null is None else np.asarray(n_null, np.int64).copy()

    def _struct(self):
        return _Chains(self.x_cur.ctypes.data, self.x_best.ctypes.data, self.d_cur.ctypes.data,
                       self.d_best.ctypes.data, self.n_accept.ctypes.data,
                       self.n_uphill.ctypes.data, self.n_null.ctypes.data)


def start_chains(net, tc, seed, n_chains, chain_ids=None):
    """x0 from the seeded sampler, objectives evaluated (the state after init)."""
    X = init_chains(net, seed, n_chains, chain_ids)
    d = np.array([objective(net, tc, x) for x in X], dtype=np.int32)
    return Chains(X, d)


def anneal(net, tc, sched, seed, chains, g0, sweeps, chain_ids=None):
    n = chains.x_cur.shape[0]
    ids = None if chain_ids is None else np.ascontiguousarray(chain_ids, dtype=np.int32)
    st = chains._struct()
    rc = lib().orc_anneal(ctypes.byref(net.s), ctypes.byref(tc.s), ctypes.byref(sched.s),
                          int(seed), int(n), _ptr(ids), int(g0), int(sweeps), ctypes.byref(st))
    if rc != ORC_OK:
        raise RuntimeError(f"orc_anneal: {rc}")
    return chains


def onehot_offsets(net):
    off = np.zeros(net.P + 1, dtype=np.int32)
    lib().orc_onehot_offsets(ctypes.byref(net.s), off.ctypes.data)
    return off


def mlp(net, X, params, target=None):
    """FP64 screening MLP.  params: W1 [D][H1], b1, W2 [H1][H2], b2, w3, b3 (any
    float arrays).  Returns y, and with a target also (loss, grads dict)."""
    X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.int8)
    B = X.shape[0]
    f = {k: np.ascontiguousarray(params[k], dtype=np.float64) for k in ("W1", "b1", "W2", "b2", "w3")}
    H1, H2 = f["W1"].shape[1], f["W2"].shape[1]
    y = np.zeros(B, np.float64)
    t = None if target is None else np.ascontiguousarray(target, dtype=np.float64)
    g = {k: np.zeros_like(v) for k, v in f.items()}
    gb3 = ctypes.c_double(0.0)
    loss = ctypes.c_double(0.0)
    grads = t is not None
    rc = lib().orc_mlp(ctypes.byref(net.s), B, X.ctypes.data, _ptr(t), H1, H2,
                       f["W1"].ctypes.data, f["b1"].ctypes.data, f["W2"].ctypes.data,
                       f["b2"].ctypes.data, f["w3"].ctypes.data, float(params["b3"]),
                       y.ctypes.data, ctypes.addressof(loss) if grads else None,
                       *( [g[k].ctypes.data for k in ("W1", "b1", "W2", "b2", "w3")] if grads
                          else [None] * 5),
                       ctypes.addressof(gb3) if grads else None)
    if rc != ORC_OK:
        raise RuntimeError(f"orc_mlp: {rc}")
    if not grads:
        return y
    g["b3"] = gb3.value
    return y, loss.value, g


def bruteforce(net, tc):
    best = ctypes.c_int32(-1)
    bx = np.zeros(net.P, dtype=np.int8)
    n = lib().orc_bruteforce(ctypes.byref(net.s), ctypes.byref(tc.s), ctypes.addressof(best),
                             bx.ctypes.data)
    if n < 0:
        raise RuntimeError(f"orc_bruteforce: {n}")
    return int(n), int(best.value), bx
