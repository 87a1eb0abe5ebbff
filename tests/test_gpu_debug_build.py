"""The debug build (libctf_debug.so, compiled with -DCTF_DEBUG) on the GPU.

Its kernels check every data-dependent texel, pixel and shared-memory index
against its buffer and record an index outside it in the device error word
(CTF_ERR_BOUNDS) instead of using it.  The debug library runs in a child
process (CTF_LIBRARY=debug), since one process loads one of the two builds:
  - the self-test reads a 32-int shared array at indices inside and outside
    it: the inside ones pass, the outside ones are recorded (and read as 0),
    and the context stays usable;
  - the parity cases of tests/debug_build_cases.py (the 128x128 plane and
    the ragged frames for every algorithm and option set, rotated quads with
    up to 54 texels per tile, the learned decode in FP16 and FP8 through
    every kernel, the batch, the texel decode and the trainer) run without a
    single record, the exact decode equals the oracle there, and every
    output equals the release library's bit for bit."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_17770_gb300 import _ctf, build  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = os.path.join(HERE, "debug_build_cases.py")


@pytest.fixture(scope="module")
def debug_lib():
    build.build()
    return build.build(debug=True)


def _child(args, timeout):
    env = dict(os.environ, CTF_LIBRARY="debug")
    r = subprocess.run([sys.executable, CASES] + args, env=env, capture_output=True, text=True, timeout=timeout,
                       cwd=os.path.dirname(HERE))
    assert r.returncode == 0, (r.stdout[-4000:], r.stderr[-4000:])
    return r.stdout.strip().splitlines()[-1]


def test_debug_selftest_records_indices_outside_the_array(debug_lib):
    out = json.loads(_child(["selftest"], 600))
    assert out["debug_build"] is True
    for index in ("0", "31", "7"):
        assert out[index]["status"] == 0, out[index]
    for index, shown in (("32", "index 32 outside [0, 32)"), ("40", "index 40 outside [0, 32)"),
                         ("-1", "index -1 outside [0, 32)")):
        assert out[index]["status"] == _ctf.CTF_ERR_BOUNDS, out[index]
        assert shown in out[index]["message"] and "the self-test" in out[index]["message"], out[index]


def test_release_library_refuses_the_bounds_selftest():
    assert not _ctf.ctf_debug_build()
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_debug_selftest_bounds(40)
    assert ei.value.status == _ctf.CTF_ERR_UNSUPPORTED
    _ctf.ctf_sync_check()


def test_debug_build_runs_the_parity_cases_without_a_record(debug_lib, tmp_path):
    import debug_build_cases as cases
    npz = tmp_path / "debug_outputs.npz"
    n = json.loads(_child([str(npz)], 1800))["cases"]
    dbg = np.load(npz)
    rel = cases.run_cases()  # this process: the release library
    assert n == len(rel) and set(dbg.files) == set(rel)
    differ = []
    for k, v in rel.items():
        a, b = np.ascontiguousarray(dbg[k]), np.ascontiguousarray(v)
        same = a.shape == b.shape and a.dtype == b.dtype and a.tobytes() == b.tobytes()
        if not same:
            differ.append(k)
    assert not differ, differ[:20]
