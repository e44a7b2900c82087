"""The C ABI library loads without a GPU and exports every entry point that
include/prd.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "prd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(prd_[A-Za-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2505_20968_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared()
    assert "prd_apply_operator" in names and "prd_solve" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_the_same_symbols():
    from paper_2505_20968_gb300 import binding
    assert sorted(binding.EXPORTS) == declared()


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: without the built library the binding raises."""
    from paper_2505_20968_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "libprd.so"))
    with pytest.raises(ImportError):
        binding.lib()


def test_errors_without_setup_and_bad_arguments():
    """Argument and ordering checks run on the host (no kernel launch)."""
    from paper_2505_20968_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.prd_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int]
    h = ctypes.c_void_p()
    rc = lib.prd_create(ctypes.byref(h), 0, 1)
    if rc != 0:
        pytest.skip("no CUDA device here: prd_create reports PRD_E_CUDA as documented")
    lib.prd_setup.argtypes = [ctypes.c_void_p]
    assert lib.prd_setup(h) == -2
