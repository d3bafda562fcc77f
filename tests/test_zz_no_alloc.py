"""rn_level_sync_noalloc: the level-end argmin and broadcast for callers that
cannot let the library allocate device memory (an application that owns all
GPU memory through its own pool or arena).  Its output must equal what the
context-owning path (rn_anneal with global_sync) produces, on two calls in a
row, bit for bit.  Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_2506_19866_gb300 import rnanneal as R
from paper_2506_19866_gb300 import synth
from tests.gpu_util import Problem

pytestmark = pytest.mark.gpu


def _level_sync_on_own_buffers(st, P, stream):
    """Run the no-allocation entry point on device buffers this test owns."""
    import torch
    n = st["x_best"].shape[0]
    row = (P + 15) // 16 * 16
    xb = torch.zeros((n, row), dtype=torch.int8, device="cuda")
    xb[:, :P] = torch.from_numpy(st["x_best"]).cuda()
    db = torch.from_numpy(st["d_best"].copy()).cuda()
    torch.cuda.synchronize()
    R.rn_level_sync_noalloc(xb, db, n, row, P, stream.cuda_stream)
    stream.synchronize()
    return xb[:, :P].cpu().numpy(), db.cpu().numpy()


def test_noalloc_level_sync_matches_context_path():
    import torch
    from paper_2506_19866_gb300 import build
    build.build()
    stream = torch.cuda.Stream()
    w = synth.make("mtb_63n_178e")
    n, L, seed = 300, 6, 41
    sync = R.schedule(8.0, 0.97, iters_per_level=L, global_sync=True)
    plain = R.schedule(8.0, 0.97, iters_per_level=L, global_sync=False)
    ctx_a, ctx_b = R.rn_create(0), R.rn_create(0)
    try:
        a = Problem(w, ctx_a)
        b = Problem(w, ctx_b)
        R.rn_init_chains(ctx_a, a.id, n, seed)
        R.rn_init_chains(ctx_b, b.id, n, seed)
        P = a.net.P
        for call in range(2):
            R.rn_anneal(ctx_a, sync, L)               # one level, ended by the context's sync
            expect = R.rn_get_chain_state(ctx_a, a.id, n)
            R.rn_anneal(ctx_b, plain, L)              # the same level without the sync ...
            got = R.rn_get_chain_state(ctx_b, b.id, n)
            xb, db = _level_sync_on_own_buffers(got, P, stream)   # ... then the no-alloc one
            np.testing.assert_array_equal(db, expect["d_best"], err_msg=f"call {call}")
            np.testing.assert_array_equal(xb, expect["x_best"], err_msg=f"call {call}")
            np.testing.assert_array_equal(got["x_cur"], expect["x_cur"])
            # the winner is the lowest objective, lowest index on ties
            win = int(np.argmin(got["d_best"]))
            assert (db == got["d_best"][win]).all() and (xb == got["x_best"][win]).all()
            got["x_best"], got["d_best"] = xb, db
            R.rn_set_chain_state(ctx_b, b.id, seed, got)
    finally:
        R.rn_destroy(ctx_a)
        R.rn_destroy(ctx_b)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2506_19866_gb300 import build
    build.build()
    x = torch.zeros(16, dtype=torch.int8, device="cuda")
    d = torch.zeros(1, dtype=torch.int32, device="cuda")
    # raw addresses, so that the library's own size check answers
    with pytest.raises(R.RNError) as e:
        R.rn_level_sync_noalloc(x.data_ptr(), d.data_ptr(), (1 << 20) + 1, 16, 8)
    assert e.value.code == R.RN_EINVAL and "1048576" in R.rn_last_error(None)


def test_noalloc_refuses_host_and_short_buffers():
    # a host pointer or a buffer shorter than n_chains rows is refused before
    # any kernel runs; the buffers are left as they were
    import torch
    from paper_2506_19866_gb300 import build
    build.build()
    x = torch.arange(64, dtype=torch.int8, device="cuda")
    d = torch.arange(4, dtype=torch.int32, device="cuda") + 5
    host = np.zeros(64, np.int8)
    with pytest.raises(R.RNError) as e:
        R.rn_level_sync_noalloc(host.ctypes.data, d.data_ptr(), 4, 16, 8)
    assert e.value.code == R.RN_EINVAL and "x_best" in R.rn_last_error(None)
    with pytest.raises(R.RNError) as e:            # rows 2^40 bytes apart: past any allocation
        R.rn_level_sync_noalloc(x.data_ptr(), d.data_ptr(), 2, 1 << 40, 8)
    assert e.value.code == R.RN_EINVAL and "allocation" in R.rn_last_error(None)
    with pytest.raises(R.RNError) as e:            # the binding's own checks on tensors
        R.rn_level_sync_noalloc(x, d, 5, 16, 8)
    assert e.value.code == R.RN_EINVAL
    with pytest.raises(R.RNError) as e:
        R.rn_level_sync_noalloc(x.cpu(), d, 4, 16, 8)
    assert e.value.code == R.RN_EINVAL
    torch.cuda.synchronize()
    assert (x.cpu().numpy() == np.arange(64)).all() and (d.cpu().numpy() == np.arange(4) + 5).all()
