"""CPU checks of the boundary: the library builds, loads without a GPU and
exports every function that include/*.h declares; host-side argument
validation answers without touching a device."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(ctf_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2506_17770_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared_functions()
    for must in ("ctf_texture_create", "ctf_texture_destroy", "ctf_filter", "ctf_filter_host",
                 "ctf_status_string", "ctf_last_error", "ctf_version"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_argument_errors_without_gpu(lib):
    from paper_2506_17770_gb300 import _ctf
    assert _ctf.ctf_status_string(-2) == "CTF_ERR_ALIGN"
    assert _ctf.ctf_status_string(0) == "CTF_OK"
    assert "sm_103a" in _ctf.ctf_version()
    # NULL texture: rejected before any CUDA call
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_filter(None, 0, 0, None, 8, 4, 0, "box", 0, None, 0, None, stream=0)
    assert ei.value.status == _ctf.CTF_ERR_ARG
    assert "NULL" in _ctf.ctf_last_error()
    # bad descriptor
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_texture_create(6, 8, 0)
    assert ei.value.status == _ctf.CTF_ERR_ARG
    # the bounded-wait self-test checks its argument before any CUDA call
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_selftest_bounded_wait(0)
    assert ei.value.status == _ctf.CTF_ERR_ARG
