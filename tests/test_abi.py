"""The C-ABI library builds, loads and exports every symbol that
include/spectra_gb.h declares; argument errors are reported without touching
a GPU."""
import ctypes
import os
import re

import pytest

from paper_2010_03817_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spectra_gb.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ["sp_create_spectrahedron", "sp_init_chains", "sp_step_billiard", "sp_step_hnr",
              "sp_step_cdhr", "sp_intersect", "sp_reflect", "sp_membership"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_errors_need_no_gpu(lib):
    lib.sp_create_spectrahedron.restype = ctypes.c_int
    lib.sp_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    assert lib.sp_create_spectrahedron(2, 3, None, 0, ctypes.byref(out)) == 1  # SP_EINVAL
    assert b"null" in lib.sp_last_error()
    assert lib.sp_intersect(None, 1, None, None, None, None, None, None, 0, None) == 1
    assert lib.sp_step_billiard(None, 1, ctypes.c_double(1.0), 10, ctypes.c_double(1e-6), 0,
                                None) == 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2010_03817_gb300 import spectra
    monkeypatch.setattr(spectra, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(spectra, "_lib", None)
    with pytest.raises(RuntimeError):
        spectra.lib()
