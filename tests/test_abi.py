"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1606_07407_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfft_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("sfft_plan_create", "sfft_execute", "sfft_signal_synthetic", "sfft_sample", "sfft_dft",
                 "sfft_classify", "sfft_plan_destroy", "sfft_signal_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_knows_every_declared_symbol():
    from paper_1606_07407_gb300 import sfft
    assert sorted(sfft.EXPORTS) == _declared()


def test_status_strings_without_gpu(lib):
    lib.sfft_status_string.restype = ctypes.c_char_p
    assert lib.sfft_status_string(0) == b"ok"
    assert lib.sfft_status_string(2) == b"not converged"


def test_invalid_arguments_rejected_without_gpu(lib):
    # argument checks run before any CUDA call
    h = ctypes.c_void_p()
    assert lib.sfft_plan_create(0, ctypes.c_int64(16), ctypes.c_int64(4), None, None, None, None,
                                ctypes.byref(h)) == 1
    assert lib.sfft_plan_create(2, ctypes.c_int64(1), ctypes.c_int64(4), None, None, None, None,
                                ctypes.byref(h)) == 1
    assert lib.sfft_execute(None, None, ctypes.c_int64(0), None, None, None, None) == 1


def test_library_is_built_for_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
