"""The C ABI library loads and exports every symbol that include/fpt.h declares (CPU only)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fpt_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2510_16172_gb300 import build

    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    names = declared_symbols()
    assert len(names) >= 15
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2510_16172_gb300 import fpt

    assert declared_symbols() <= set(fpt._SIGS), declared_symbols() - set(fpt._SIGS)
    fpt.library()


def test_default_params_without_gpu(lib_path):
    from paper_2510_16172_gb300 import fpt

    p = fpt.default_params()
    assert p.max_iters == 64 and p.fp_iters == 1 and p.polish == 1
    assert abs(p.tol_step - 1e-4) < 1e-9 and abs(p.solved_tol - 1e-5) < 1e-10


def test_missing_library_fails_loudly(tmp_path):
    from paper_2510_16172_gb300 import fpt

    with pytest.raises(fpt.FptLibraryMissing):
        fpt._lib_backup = fpt._lib
        try:
            fpt._lib = None
            fpt.library(str(tmp_path / "nope.so"))
        finally:
            fpt._lib = fpt._lib_backup
