"""The C-ABI library builds, loads and exports every entry point that
include/afps.h declares; calls that need no GPU behave as documented."""
import ctypes
import os
import re

import pytest

from paper_2208_08795_gb300 import afps as B
from paper_2208_08795_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    with open(os.path.join(ROOT, "include", "afps.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(afps_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return B.load()


def test_header_lists_entry_points():
    names = header_functions()
    assert "afps_sample" in names and "afps_sample_batched" in names
    assert sorted(B.EXPORTS) == names


def test_every_declared_symbol_is_exported(lib):
    for name in header_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_null_context_is_rejected(lib):
    assert lib.afps_sample(None, None, 1, 1, 1, 0, 0, None, None) == B.AFPS_ERR_INVALID_ARG
    assert lib.afps_sync(None, None) == B.AFPS_ERR_INVALID_ARG
    assert lib.afps_last_error(None) == b"NULL context"
    assert lib.afps_launch_count(None) == 0
    lib.afps_destroy(None)  # no-op


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    cfg = B.afps_config(0, 0, 0, None)
    assert lib.afps_create(ctypes.byref(h), ctypes.byref(cfg)) == B.AFPS_ERR_CUDA
    assert h.value is None


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(B.AfpsLibraryError):
        B.load(str(tmp_path / "nope.so"))
    monkeypatch.setattr(B, "_lib", None)


def test_python_constants_match_the_header():
    """Every error code, flag, method and key the header defines has the
    same value in the binding."""
    import re
    here = os.path.dirname(os.path.abspath(__file__))
    text = open(os.path.join(here, "..", "include", "afps.h")).read()
    defs = dict(re.findall(r"#define (AFPS_[A-Z0-9_]+) \(?(-?(?:0x)?[0-9a-fA-F]+)u?\)?", text))
    checked = 0
    for name, val in defs.items():
        if name.startswith(("AFPS_ERR_", "AFPS_FLAG_", "AFPS_METHOD_", "AFPS_KEY_")):
            assert hasattr(B, name), name
            assert getattr(B, name) == int(val, 0), name
            checked += 1
    assert checked >= 12
