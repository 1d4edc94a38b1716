"""The C-ABI library builds for sm_103a, loads on a machine without a GPU and
exports every function that include/*.h declares (no compute is called)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(tnmc_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("no CUDA toolkit")
    from paper_2509_23945_gb300 import build_lib
    path = build_lib.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tnmc_create", "tnmc_slice_update", "tnmc_sweep", "tnmc_destroy", "tnmc_slice_logz"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2509_23945_gb300 import tnmc
    bound = {name for name, _, _ in tnmc.SIGNATURES}
    assert declared_functions() <= bound, declared_functions() - bound


def test_binding_refuses_without_library(tmp_path):
    from paper_2509_23945_gb300 import tnmc
    saved = tnmc._lib
    tnmc._lib = None
    try:
        with pytest.raises(RuntimeError):
            tnmc.load_library(str(tmp_path / "missing.so"))
    finally:
        tnmc._lib = saved
