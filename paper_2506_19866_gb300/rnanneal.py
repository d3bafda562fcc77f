"""Python binding of librnanneal.so (include/rnanneal.h), argument marshalling only.

Every function has the name of the C entry point it calls and raises
RNError on a negative return code.  Host arrays are numpy arrays; device
arrays (rn_evaluate_device) are torch CUDA tensors or raw device addresses.
There is no fallback: if the library is missing, loading fails with an
ImportError naming the build step.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librnanneal.so")

RN_OK, RN_EINVAL, RN_ECONSTRAINT, RN_ENOMEM, RN_ECUDA, RN_ETIMEOUT, RN_ESTATE, \
    RN_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
_NAMES = {-1: "RN_EINVAL", -2: "RN_ECONSTRAINT", -3: "RN_ENOMEM", -4: "RN_ECUDA",
          -5: "RN_ETIMEOUT", -6: "RN_ESTATE", -7: "RN_EUNSUPPORTED"}

# every entry point the header declares, with its ctypes signature
_c_int, _c_i32, _c_i64, _c_u64, _vp = (ctypes.c_int, ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_uint64, ctypes.c_void_p)


class rn_schedule(ctypes.Structure):
    _fields_ = [("T0", ctypes.c_double), ("alpha", ctypes.c_double),
                ("iters_per_level", ctypes.c_int64), ("reset_to_best", ctypes.c_int32),
                ("global_sync", ctypes.c_int32), ("early_reject", ctypes.c_int32),
                ("sync_group", ctypes.c_int32)]


SIGNATURES = {
    "rn_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _vp]),
    "rn_destroy": (_c_int, [_vp]),
    "rn_last_error": (ctypes.c_char_p, [_vp]),
    "rn_load_network": (_c_int, [_vp, _c_i32, _c_i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rn_load_timecourse": (_c_int, [_vp, _c_i32, _c_i32, _c_i32, _vp, _vp, _vp, _vp]),
    "rn_init_chains": (_c_int, [_vp, _c_i32, _c_i32, _c_u64, _vp]),
    "rn_anneal": (_c_int, [_vp, ctypes.POINTER(rn_schedule), _c_i64]),
    "rn_get_best": (_c_int, [_vp, _c_i32, _vp, _vp, _vp]),
    "rn_evaluate": (_c_int, [_vp, _c_i32, _c_i32, _vp, _vp, _vp]),
    "rn_evaluate_device": (_c_int, [_vp, _c_i32, _c_i32, _vp, _vp, _vp]),
    "rn_n_params": (_c_int, [_vp, _c_i32, _vp]),
    "rn_get_chain_state": (_c_int, [_vp, _c_i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rn_set_chain_state": (_c_int, [_vp, _c_i32, _c_i32, _c_u64, _vp, _vp, _vp, _vp, _vp,
                                    _c_i64]),
    "rn_prepare_schedule": (_c_int, [_vp, ctypes.POINTER(rn_schedule), _c_i64]),
    "rn_get_stats": (_c_int, [_vp, _c_i32, _vp]),
    "rn_selftest_wait": (_c_int, [_vp]),
    "rn_launch_count": (_c_int, [_vp, _vp]),
    "rn_batch_config": (_c_int, [_vp, _vp, _vp]),
    "rn_batch_tune": (_c_int, [_vp, _c_i32]),
    "rn_set_update_scheme": (_c_int, [_vp, _c_i32, _c_i32, _vp]),
    "rn_level_sync_noalloc": (_c_int, [_vp, _vp, _c_i32, _c_i64, _c_i32, _vp]),
    "rn_mlp_create": (_c_int, [_vp, _c_i32, _c_i32, _c_i32, _c_i64, _vp, _vp]),
    "rn_mlp_set_weights": (_c_int, [_vp, _c_i32, _vp, _vp, _vp, _vp, _vp, ctypes.c_float]),
    "rn_mlp_get_weights": (_c_int, [_vp, _c_i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rn_mlp_forward": (_c_int, [_vp, _c_i32, _c_i32, _vp, _vp]),
    "rn_mlp_gradients": (_c_int, [_vp, _c_i32, _c_i32, _vp, _vp] + [_vp] * 7),
    "rn_mlp_add_samples": (_c_int, [_vp, _c_i32, _c_i32, _vp, _vp, _vp]),
    "rn_mlp_log_chains": (_c_int, [_vp, _c_i32, _vp]),
    "rn_mlp_train": (_c_int, [_vp, _c_i32, _c_i32, _c_i32, ctypes.c_float, _c_u64, _vp]),
    "rn_anneal_screened": (_c_int, [_vp, _c_i32, ctypes.POINTER(rn_schedule), _c_i32, _c_i32,
                                    ctypes.c_double, _c_i64]),
    "rn_mlp_set_hidden_mode": (_c_int, [_vp, _c_i32, _c_i32]),
    "rn_synchronize": (_c_int, [_vp]),
}


class RNError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load librnanneal.so and declare its signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run __graft_entry__.build() (or "
                              f"python -m paper_2506_19866_gb300.build) first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(ctx, rc):
    if rc != RN_OK:
        msg = load_library().rn_last_error(ctx)
        raise RNError(rc, msg.decode() if msg else "")


def _arr(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data


def _dev(t):
    if t is None:
        return None
    return int(t) if isinstance(t, int) else int(t.data_ptr())


def _dev_checked(t, dtype_name, min_numel, name):
    """Device address of a torch CUDA tensor after checking its device, dtype,
    contiguity and size (a raw integer address is passed through; the library
    checks it against its allocation)."""
    if t is None or isinstance(t, int):
        return _dev(t)
    if not getattr(t, "is_cuda", False):
        raise RNError(RN_EINVAL, f"{name}: a CUDA tensor is required")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise RNError(RN_EINVAL, f"{name}: dtype {t.dtype}, expected torch.{dtype_name}")
    if not t.is_contiguous():
        raise RNError(RN_EINVAL, f"{name}: must be contiguous")
    if t.numel() < min_numel:
        raise RNError(RN_EINVAL, f"{name}: {t.numel()} elements, at least {min_numel} needed")
    return int(t.data_ptr())


def rn_create(device: int = 0, stream=None):
    h = _vp()
    s = None if stream is None else int(stream)
    _check(None, load_library().rn_create(ctypes.byref(h), int(device), s))
    return h.value


def rn_destroy(ctx):
    load_library().rn_destroy(ctx)


def rn_last_error(ctx):
    return load_library().rn_last_error(ctx).decode()


def rn_load_network(ctx, src, dst, fast, frozen=None, frozen_val=None):
    src, dst = _arr(src, np.int32), _arr(dst, np.int32)
    fast = _arr(fast, np.uint8)
    frozen, frozen_val = _arr(frozen, np.uint8), _arr(frozen_val, np.int8)
    out = ctypes.c_int32(-1)
    _check(ctx, load_library().rn_load_network(ctx, fast.size, src.size, _p(src), _p(dst),
                                               _p(fast), _p(frozen), _p(frozen_val),
                                               ctypes.byref(out)))
    return out.value


def rn_load_timecourse(ctx, net, init, ref, observed, knockout=None):
    init, ref, observed = _arr(init, np.uint8), _arr(ref, np.uint8), _arr(observed, np.uint8)
    knockout = _arr(knockout, np.uint8)
    C, T = ref.shape[0], ref.shape[1]
    _check(ctx, load_library().rn_load_timecourse(ctx, int(net), C, T, _p(init), _p(knockout),
                                                  _p(ref), _p(observed)))


def rn_init_chains(ctx, net, n_chains, seed, x0=None):
    x0 = _arr(x0, np.int8)
    _check(ctx, load_library().rn_init_chains(ctx, int(net), int(n_chains), int(seed), _p(x0)))


def schedule(T0, alpha, iters_per_level=1, reset_to_best=False, global_sync=False,
             early_reject=False, sync_group=0):
    return rn_schedule(float(T0), float(alpha), int(iters_per_level), int(bool(reset_to_best)),
                       int(bool(global_sync)), int(bool(early_reject)), int(sync_group))


def rn_anneal(ctx, sched: rn_schedule, sweeps):
    _check(ctx, load_library().rn_anneal(ctx, ctypes.byref(sched), int(sweeps)))


def rn_n_params(ctx, net):
    out = ctypes.c_int32(0)
    _check(ctx, load_library().rn_n_params(ctx, int(net), ctypes.byref(out)))
    return out.value


def rn_get_best(ctx, net):
    P = rn_n_params(ctx, net)
    x = np.zeros(P, dtype=np.int8)
    score, chain = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(ctx, load_library().rn_get_best(ctx, int(net), _p(x), ctypes.byref(score),
                                           ctypes.byref(chain)))
    return x, score.value, chain.value


def rn_evaluate(ctx, net, x, traj_shape=None):
    """x: [n][P] int8.  traj_shape (C, T, N) requests trajectories."""
    x = _arr(np.atleast_2d(x), np.int8)
    n = x.shape[0]
    score = np.zeros(n, dtype=np.int32)
    traj = None if traj_shape is None else np.zeros((n, *traj_shape), dtype=np.uint8)
    _check(ctx, load_library().rn_evaluate(ctx, int(net), n, _p(x), _p(score), _p(traj)))
    return score if traj is None else (score, traj)


def rn_evaluate_device(ctx, net, n, x_dev, score_dev, traj_dev=None):
    """x_dev [n][P] int8, score_dev [n] int32, traj_dev [n][C][T][N] uint8 or
    None: torch CUDA tensors (checked here) or raw device addresses."""
    n = int(n)
    P = rn_n_params(ctx, net) if n > 0 else 0
    x = _dev_checked(x_dev, "int8", n * P, "x_dev") if n > 0 else _dev(x_dev)
    s = _dev_checked(score_dev, "int32", n, "score_dev") if n > 0 else _dev(score_dev)
    t = _dev_checked(traj_dev, "uint8", n, "traj_dev") if n > 0 else _dev(traj_dev)
    _check(ctx, load_library().rn_evaluate_device(ctx, int(net), n, x, s, t))


def rn_get_chain_state(ctx, net, n_chains):
    P = rn_n_params(ctx, net)
    st = dict(x_cur=np.zeros((n_chains, P), np.int8), d_cur=np.zeros(n_chains, np.int32),
              x_best=np.zeros((n_chains, P), np.int8), d_best=np.zeros(n_chains, np.int32),
              counters=np.zeros((n_chains, 3), np.int64))
    step = ctypes.c_int64(0)
    _check(ctx, load_library().rn_get_chain_state(ctx, int(net), _p(st["x_cur"]), _p(st["d_cur"]),
                                                  _p(st["x_best"]), _p(st["d_best"]),
                                                  _p(st["counters"]), ctypes.byref(step)))
    st["step"] = step.value
    return st


def rn_set_chain_state(ctx, net, seed, st):
    xc, xb = _arr(st["x_cur"], np.int8), _arr(st["x_best"], np.int8)
    dc, db = _arr(st["d_cur"], np.int32), _arr(st["d_best"], np.int32)
    cnt = _arr(st["counters"], np.int64)
    _check(ctx, load_library().rn_set_chain_state(ctx, int(net), xc.shape[0], int(seed), _p(xc),
                                                  _p(dc), _p(xb), _p(db), _p(cnt),
                                                  int(st["step"])))


def rn_synchronize(ctx):
    _check(ctx, load_library().rn_synchronize(ctx))


def rn_prepare_schedule(ctx, sched: rn_schedule, total_steps):
    _check(ctx, load_library().rn_prepare_schedule(ctx, ctypes.byref(sched), int(total_steps)))


def rn_get_stats(ctx, net):
    """Accepted, uphill (dE > 0) and null moves summed over a network's chains,
    the number of chains and the next global step."""
    s = np.zeros(5, np.int64)
    _check(ctx, load_library().rn_get_stats(ctx, int(net), _p(s)))
    return dict(accepted=int(s[0]), uphill=int(s[1]), null=int(s[2]), chains=int(s[3]),
                step=int(s[4]))


def rn_selftest_wait(ctx):
    """Run one device-side wait that must give up; raises RNError with
    RN_ETIMEOUT when the failure path works (see the header)."""
    _check(ctx, load_library().rn_selftest_wait(ctx))


def rn_launch_count(ctx):
    out = ctypes.c_int64(0)
    _check(ctx, load_library().rn_launch_count(ctx, ctypes.byref(out)))
    return out.value


def rn_batch_config(ctx):
    """Networks, warps per block, large-region (shared-memory or hybrid) networks,
    graph replay, hybrid networks, candidate in use, kernels per batched launch
    (phases), trial ms of the candidates."""
    info = np.zeros(7, np.int32)
    ms = np.zeros(10, np.float64)
    _check(ctx, load_library().rn_batch_config(ctx, _p(info), _p(ms)))
    return dict(networks=int(info[0]), warps_per_block=int(info[1]),
                shared_path_networks=int(info[2]), graph=bool(info[3]),
                hybrid_networks=int(info[4]), config=int(info[5]), phases=int(info[6]),
                trial_ms=ms.tolist())


def rn_set_update_scheme(ctx, net, scheme, selected=None):
    """0: priority updating (default); 1: synchronous updating; 2: asynchronous
    updating with selected[C][T] the node that may move at each step (Section 2.2)."""
    sel = None if selected is None else _arr(selected, np.int32)
    _check(ctx, load_library().rn_set_update_scheme(ctx, int(net), int(scheme), _p(sel)))


def rn_batch_tune(ctx, config):
    """Pin the batched launch to candidate 0..9, or autotune again with -1."""
    _check(ctx, load_library().rn_batch_tune(ctx, int(config)))


def rn_level_sync_noalloc(x_best_dev, d_best_dev, n_chains, row_bytes, n_params, stream=None):
    """Level-end argmin + broadcast on caller-owned device buffers; allocates nothing."""
    s = None if stream is None else int(stream)
    n, row, P = int(n_chains), int(row_bytes), int(n_params)
    span = (n - 1) * row + P if n > 0 else 0
    x = _dev_checked(x_best_dev, "int8", span, "x_best")
    d = _dev_checked(d_best_dev, "int32", max(n, 0), "d_best")
    _check(None, load_library().rn_level_sync_noalloc(x, d, n, row, P, s))


# ---- learned proposal screen -------------------------------------------------

def rn_mlp_create(ctx, net, h1=512, h2=512, capacity=1 << 20):
    """Returns (screen id, one-hot width D)."""
    mid, D = ctypes.c_int32(-1), ctypes.c_int32(0)
    _check(ctx, load_library().rn_mlp_create(ctx, int(net), int(h1), int(h2), int(capacity),
                                             ctypes.byref(mid), ctypes.byref(D)))
    return mid.value, D.value


_WEIGHTS = ("W1", "b1", "W2", "b2", "w3")


def rn_mlp_set_weights(ctx, mlp, params):
    """params: dict W1 [D][h1], b1, W2 [h1][h2], b2, w3, b3."""
    a = {k: _arr(params[k], np.float32) for k in _WEIGHTS}
    _check(ctx, load_library().rn_mlp_set_weights(ctx, int(mlp), *[_p(a[k]) for k in _WEIGHTS],
                                                  float(params["b3"])))


def rn_mlp_get_weights(ctx, mlp, D, h1, h2):
    out = dict(W1=np.zeros((D, h1), np.float32), b1=np.zeros(h1, np.float32),
               W2=np.zeros((h1, h2), np.float32), b2=np.zeros(h2, np.float32),
               w3=np.zeros(h2, np.float32))
    b3 = np.zeros(1, np.float32)
    _check(ctx, load_library().rn_mlp_get_weights(ctx, int(mlp), *[_p(out[k]) for k in _WEIGHTS],
                                                  _p(b3)))
    out["b3"] = float(b3[0])
    return out


def rn_mlp_forward(ctx, mlp, x):
    x = _arr(np.atleast_2d(x), np.int8)
    y = np.zeros(x.shape[0], np.float32)
    _check(ctx, load_library().rn_mlp_forward(ctx, int(mlp), x.shape[0], _p(x), _p(y)))
    return y


def rn_mlp_gradients(ctx, mlp, x, target, D, h1, h2):
    """Returns (loss, grads dict with the keys of rn_mlp_get_weights)."""
    x = _arr(np.atleast_2d(x), np.int8)
    t = _arr(target, np.float32)
    g = dict(W1=np.zeros((D, h1), np.float32), b1=np.zeros(h1, np.float32),
             W2=np.zeros((h1, h2), np.float32), b2=np.zeros(h2, np.float32),
             w3=np.zeros(h2, np.float32))
    loss, gb3 = ctypes.c_float(0), ctypes.c_float(0)
    _check(ctx, load_library().rn_mlp_gradients(ctx, int(mlp), x.shape[0], _p(x), _p(t),
                                                ctypes.byref(loss),
                                                *[_p(g[k]) for k in _WEIGHTS],
                                                ctypes.byref(gb3)))
    g["b3"] = gb3.value
    return loss.value, g


def rn_mlp_add_samples(ctx, mlp, x, target):
    x = _arr(np.atleast_2d(x), np.int8)
    t = _arr(target, np.float32)
    count = ctypes.c_int64(0)
    _check(ctx, load_library().rn_mlp_add_samples(ctx, int(mlp), x.shape[0], _p(x), _p(t),
                                                  ctypes.byref(count)))
    return count.value


def rn_mlp_log_chains(ctx, mlp):
    count = ctypes.c_int64(0)
    _check(ctx, load_library().rn_mlp_log_chains(ctx, int(mlp), ctypes.byref(count)))
    return count.value


def rn_mlp_train(ctx, mlp, steps, batch=4096, lr=1e-3, seed=0):
    loss = ctypes.c_float(0)
    _check(ctx, load_library().rn_mlp_train(ctx, int(mlp), int(steps), int(batch), float(lr),
                                            int(seed), ctypes.byref(loss)))
    return loss.value


def rn_anneal_screened(ctx, mlp, sched: rn_schedule, sweeps, K=32, top=2, eps=0.0):
    _check(ctx, load_library().rn_anneal_screened(ctx, int(mlp), ctypes.byref(sched), int(K),
                                                  int(top), float(eps), int(sweeps)))


def rn_mlp_set_hidden_mode(ctx, mlp, mode):
    """1: the screened step's layer-2 input rows go through device memory
    (propose kernel writes, TMA reads; the default); 0: formed inside the GEMM."""
    _check(ctx, load_library().rn_mlp_set_hidden_mode(ctx, int(mlp), int(mode)))
