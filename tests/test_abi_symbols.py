"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/qtt.h declares (no GPU needed: nothing is called but
qtt_version and qtt_last_error, which touch no device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qtt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?[\s\*])(qtt_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2301_13339_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_parses():
    names = declared_functions()
    for n in ("qtt_decompose", "qtt_conv_sinc", "qtt_round", "qtt_to_full", "qtt_conv_adjoint",
              "qtt_get_ranks", "qtt_free", "qtt_last_error"):
        assert n in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in qtt.h but not exported: {missing}"


def test_binding_list_matches_header():
    import paper_2301_13339_gb300 as q
    assert set(q.EXPORTED_SYMBOLS) <= set(declared_functions())
    public = [n for n in declared_functions() if not n.startswith("qtt_debug_")]
    missing = sorted(set(public) - set(q.EXPORTED_SYMBOLS))
    assert not missing, f"no binding for {missing}"


def test_version_string_without_device(lib):
    lib.qtt_version.restype = ctypes.c_char_p
    lib.qtt_last_error.restype = ctypes.c_char_p
    assert lib.qtt_version().decode().startswith("qtt")
    assert isinstance(lib.qtt_last_error(), bytes)
