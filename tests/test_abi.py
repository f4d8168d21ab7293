"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/nlsp.h declares; the Python binding covers them all."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^NLSP_API[^;(]*?\b(nlsp_\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2601_20174_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    assert len(names) >= 20 and len(set(names)) == len(names)


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib_path):
    from paper_2601_20174_gb300 import _lib
    assert set(_declared()) <= set(_lib.SIGNATURES), set(_declared()) - set(_lib.SIGNATURES)
    lib = _lib.load()
    assert lib.nlsp_status_string(-3).decode() == "NLSP_ERR_NOT_SPD"


def test_fails_loudly_without_gpu_on_create(lib_path):
    # Without a device the context cannot be created: an error status, no crash.
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2601_20174_gb300 import _lib
    h = ctypes.c_void_p()
    st = _lib.load().nlsp_create(ctypes.byref(h), 0, None)
    assert st in (_lib.NLSP_ERR_INVALID, _lib.NLSP_ERR_CUDA)
