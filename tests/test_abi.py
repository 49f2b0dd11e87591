"""The C ABI library loads and exports every entry point that include/vc.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:int|const char\s*\*|void)\s*\*?\s*(vc_\w+)\s*\(", text, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_10402_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_symbols()
    for want in ("vc_mvc", "vc_pvc", "vc_mvc_batch"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_names_match_header():
    import paper_2204_10402_gb300 as vc
    assert set(declared_symbols()) == set(vc.EXPORTED)


def test_host_only_calls(lib):
    lib.vc_version.restype = ctypes.c_int
    assert lib.vc_version() >= 100
    lib.vc_strerror.restype = ctypes.c_char_p
    assert lib.vc_strerror(-1) == b"VC_EINVAL"
    assert lib.vc_strerror(0) == b"VC_OK"
