"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/rnanneal.h (no compute calls: runs without a GPU)."""
import os
import re
import subprocess

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


def test_header_is_plain_c_and_cxx():
    for cmd in (["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                 "-x", "c", HEADER],
                ["g++", "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                 "-x", "c++", HEADER]):
        subprocess.check_call(cmd)


def test_c_program_links_every_entry_point(lib, tmp_path):
    # a C program that takes the address of every declared entry point links
    # against the library: the names have C linkage and the declarations are C
    names = declared_entry_points()
    src = tmp_path / "abi_link.c"
    src.write_text('#include "rnanneal.h"\nint main(void) {\n    void (*fns[])(void) = {\n'
                   + ",\n".join(f"        (void (*)(void))&{n}" for n in names)
                   + "\n    };\n    return (int)(sizeof fns / sizeof fns[0]) == %d ? 0 : 1;\n}\n"
                   % len(names))
    cuda_lib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER),
                           str(src), "-L", os.path.dirname(R.LIB_PATH), "-lrnanneal",
                           f"-Wl,-rpath-link,{cuda_lib}", "-o", str(tmp_path / "abi_link")])


def test_product_never_loads_the_oracle():
    # the package and its kernels hold no import, library name or symbol of the
    # oracle: the product path cannot route through it
    pkg = os.path.join(B.ROOT, "paper_2506_19866_gb300")
    pattern = re.compile(r"import\s+oracle|from\s+oracle|liboracle|\borc_[a-z]")
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(root, f)) as fh:
                    assert not pattern.search(fh.read()), os.path.join(root, f)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no fallback: without the built library the binding raises
    monkeypatch.setattr(R, "_lib", None)
    with pytest.raises(ImportError):
        R.load_library(str(tmp_path / "librnanneal.so"))
