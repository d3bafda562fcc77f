"""Host-side logic of the kernels, checked without a GPU.
- The block path's table layout, built by the library on the host: every edge
  in exactly one entry of its node's lane and slot, edge_pos naming that entry,
  every code address inside the block's code region, and, on the register
  variant's two copies of the state codes, a code gather with fewer wavefronts
  than any placement over one copy could reach (tests/layout_check.cu reads the
  layout through the library's own builder).
- GetCandidate's choice of the new value (tests/candidate_check.cu)."""
import os
import subprocess

import numpy as np
import pytest

from paper_2506_19866_gb300 import build as B
from paper_2506_19866_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    B.build()
    out = tmp_path_factory.mktemp("layout") / "layout_check"
    lib_dir = os.path.join(B.ROOT, "paper_2506_19866_gb300")
    subprocess.check_call([B._nvcc(), *B.ARCH, "-std=c++17", "-O2", "-I", os.path.join(B.ROOT, "include"),
                           os.path.join(HERE, "layout_check.cu"), "-o", str(out),
                           "-L", lib_dir, "-lrnanneal", "-Xlinker", f"-rpath={lib_dir}"])
    return str(out)


def _run(checker, tmp_path, w):
    f = tmp_path / "net.bin"
    with open(f, "wb") as fh:
        np.array([w.N, len(w.src)], np.int32).tofile(fh)
        np.asarray(w.src, np.int32).tofile(fh)
        np.asarray(w.dst, np.int32).tofile(fh)
    r = subprocess.run([checker, str(f)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    v = r.stdout.split()
    return dict(zip(v[0::2], (int(x) for x in v[1::2])))


def test_two_copies_cut_the_code_gather(checker, tmp_path):
    # the 2000-node, 16-condition network: 8 nodes per thread, register variant
    s = _run(checker, tmp_path, synth.make("n2000_c16_t33"))
    assert s["supported"] == 1 and s["npl"] == 8 and s["two_copies"] == 1
    assert s["wavefronts"] < s["lower_bound_one_copy"]
    assert s["wavefronts"] <= 1.15 * s["rows"]


@pytest.mark.parametrize("seed,n_nodes,lam,cap", [(61, 700, 5.0, 20), (64, 1200, 27.0, 31),
                                                  (66, 600, 20.0, 31), (62, 513, 4.0, 24),
                                                  (65, 2900, 2.0, 8), (67, 90, 24.0, 31)])
def test_block_layouts_place_every_edge_once(checker, tmp_path, seed, n_nodes, lam, cap):
    # register variants (2, 4, 6 nodes per thread), the shared-memory variant
    # (12 per thread: one copy) and a small network of in-degree above 16
    w = synth.random_network(seed, n_nodes, lam=lam, cap=cap, n_cond=2, n_times=4, obs_frac=0.5)
    s = _run(checker, tmp_path, w)
    assert s["supported"] == 1 and s["lanes"] == 256
    assert s["two_copies"] == (1 if s["npl"] <= 8 else 0)
    assert s["wavefronts"] >= s["rows"]


def test_candidate_value_choice(tmp_path):
    # GetCandidate's branch-free choice of the new value (pick_alternative)
    # against a walk over the listed domains, every case that can arise
    exe = tmp_path / "candidate_check"
    subprocess.check_call([B._nvcc(), *B.ARCH, "-std=c++17", "-O2",
                           os.path.join(HERE, "candidate_check.cu"), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert int(r.stdout.split()[1]) > 1_000_000
