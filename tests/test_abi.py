"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/rnanneal.h (no compute calls: runs without a GPU)."""
import os
import re

import pytest

from paper_2506_19866_gb300 import build as B
from paper_2506_19866_gb300 import rnanneal as R

HEADER = os.path.join(B.ROOT, "include", "rnanneal.h")


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rn_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return R.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert "rn_anneal" in names and "rn_evaluate" in names and len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    assert set(R.SIGNATURES) == set(declared_entry_points())


def test_library_targets_sm103a(lib):
    # the only device code in the library is sm_103a SASS (checked through the
    # build flags, not by reading the binary)
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_create_reports_missing_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(R.RNError) as ei:
        R.rn_create(0)
    assert ei.value.code == R.RN_ECUDA
    assert R.rn_last_error(None)
