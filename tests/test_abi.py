"""The C ABI library loads on a machine without a GPU and exports every function that
include/woodelf.h declares; error paths that need no device report cleanly."""
import ctypes
import os
import re

import paper_2511_09376_gb300 as wdf

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "woodelf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wdf_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 12
    lib = ctypes.CDLL(wdf.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_null_argument_errors():
    assert "sm_103a" in wdf.version()
    lib = ctypes.CDLL(wdf.library_path())
    lib.wdf_last_error.restype = ctypes.c_char_p
    assert lib.wdf_ctx_create(0, None) == 1
    assert b"null" in lib.wdf_last_error()
    assert lib.wdf_explain(None, None, 0, 0, 1, None, 0, None) == 1
    assert lib.wdf_ensemble_info(None, None) == 1
