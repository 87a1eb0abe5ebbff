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


def _fnv1a(data):
    h = 14695981039346656037
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _texture_file(mode, w, h, lat, payload, version=1):
    import struct
    body = b"CTFTEX01" + struct.pack("<I7i", version, mode, w, h, *lat) + payload
    return body + struct.pack("<Q", _fnv1a(body))


def test_malformed_texture_checkpoints_are_refused_without_gpu(lib, tmp_path):
    """ctf_checkpoint_load reads and checks the whole file before any device
    work: a missing file, a foreign file, a bad checksum, another version,
    impossible sizes, a payload of the wrong length and a weight that FP16
    cannot hold are each refused."""
    import struct
    import numpy as np
    from paper_2506_17770_gb300 import _ctf
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_checkpoint_load(str(tmp_path / "missing.ctftex"))
    assert ei.value.status == _ctf.CTF_ERR_ARG
    # an FP16 texture with 1x1 latent grids: 8 + 8 + 1024 + 64 + 4096 + 64 + 256 + 4 floats
    n = 8 + 8 + 1024 + 64 + 4096 + 64 + 256 + 4
    good = np.zeros(n, np.float32).tobytes()
    bad_value = np.zeros(n, np.float32)
    bad_value[16] = 0.1  # w1[0][0] is not an FP16 number
    cases = {
        "foreign": b"\x7fELF" + bytes(100),
        "checksum": _texture_file(1, 64, 64, (1, 1, 1, 1), good)[:-1] + b"\x00",
        "version": _texture_file(1, 64, 64, (1, 1, 1, 1), good, version=2),
        "mode": _texture_file(7, 64, 64, (1, 1, 1, 1), good),
        "block_sides": _texture_file(0, 6, 8, (0, 0, 0, 0), bytes(16)),
        "block_length": _texture_file(0, 8, 8, (0, 0, 0, 0), bytes(24)),
        "latent_side": _texture_file(1, 64, 64, (0, 1, 1, 1), good),
        "length": _texture_file(1, 64, 64, (1, 1, 1, 1), good[:-4]),
        "value": _texture_file(1, 64, 64, (1, 1, 1, 1), bad_value.tobytes()),
    }
    for name, raw in cases.items():
        path = tmp_path / (name + ".ctftex")
        path.write_bytes(raw)
        with pytest.raises(_ctf.CtfError) as ei:
            _ctf.ctf_checkpoint_load(str(path))
        assert ei.value.status == _ctf.CTF_ERR_CORRUPT, (name, _ctf.ctf_last_error())


def test_mlp_train_checks_its_arguments_without_gpu(lib):
    from paper_2506_17770_gb300 import _ctf
    desc = _ctf.train_desc(((8, 8), (4, 4)), batch=64, total_steps=1)
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_mlp_train(None, desc, _ctf.CTF_EVAL_BLOCK)
    assert ei.value.status == _ctf.CTF_ERR_ARG


def test_every_device_allocation_goes_through_the_counted_routine():
    """The allocation test hooks (and the no-allocation entry point's test,
    which reads the counter) rely on this: no source file of the library
    calls a CUDA allocator or cudaFree except the one counted routine."""
    csrc = os.path.join(ROOT, "paper_2506_17770_gb300", "csrc")
    pat = re.compile(r"\b(cudaMalloc\w*|cudaFree\w*|cudaHostAlloc|cuMem(Alloc|Free)\w*)\s*\(")
    offenders = []
    for path in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))
                       + glob.glob(os.path.join(csrc, "*.h"))):
        src = open(path).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        src = re.sub(r'"(\\.|[^"\\])*"', '""', src)
        for m in pat.finditer(src):
            offenders.append((os.path.basename(path), m.group(1), src[:m.start()].count("\n") + 1))
    allowed = [o for o in offenders if o[0] == "ctf_api.cu" and o[1] in ("cudaMalloc", "cudaFree")]
    assert len(allowed) == 2, offenders
    assert not [o for o in offenders if o not in allowed], offenders


def test_allocation_hook_checks_its_arguments_without_gpu(lib):
    from paper_2506_17770_gb300 import _ctf
    for skip, n in ((0, -1), (-1, 1)):
        with pytest.raises(_ctf.CtfError) as ei:
            _ctf.ctf_debug_fail_allocations(n, skip=skip)
        assert ei.value.status == _ctf.CTF_ERR_ARG
    _ctf.ctf_debug_fail_allocations(0)
    assert _ctf.ctf_debug_device_allocations() >= 0
    assert _ctf.ctf_debug_live_allocations() >= 0


def test_debug_build_exports_the_same_entry_points_without_gpu(lib):
    """The debug library (index checks in every kernel) builds from the same
    sources, exports every declared function and says which build it is;
    the release library refuses the bounds self-test before any CUDA call."""
    from paper_2506_17770_gb300 import _ctf, build
    dbg = ctypes.CDLL(build.build(debug=True))
    missing = [n for n in _declared_functions() if not hasattr(dbg, n)]
    assert not missing, missing
    assert dbg.ctf_debug_build() == 1
    assert lib.ctf_debug_build() == 0
    assert _ctf.ctf_status_string(_ctf.CTF_ERR_BOUNDS) == "CTF_ERR_BOUNDS"
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_debug_selftest_bounds(40)
    assert ei.value.status == _ctf.CTF_ERR_UNSUPPORTED


def test_debug_index_checks_cover_the_kernels_sources():
    """Every translation unit with kernels that index texels, pixels or
    shared tables goes through the debug build's check (ck) somewhere, and
    the release definition of ck is the index itself."""
    csrc = os.path.join(ROOT, "paper_2506_17770_gb300", "csrc")
    for name in ("ctf_exact_tile.cuh", "ctf_select.cuh", "ctf_mlp_chain.cuh", "ctf_mlp_ws2.cu", "ctf_mlp_ext.cu",
                 "ctf_bicubic.cu", "ctf_batch.cu", "ctf_train.cu", "ctf_device.cuh"):
        assert "ck(" in open(os.path.join(csrc, name)).read(), name
    dbg = open(os.path.join(csrc, "ctf_debug.cuh")).read()
    release = dbg[dbg.index("#else"):dbg.index("#endif")]
    assert "return i;" in release and "atomic" not in release
