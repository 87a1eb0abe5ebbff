"""ctf_filter_host_noalloc: the host-buffer filter for callers that cannot let
the library allocate device memory.

Such callers (a renderer or plug-in whose video memory is reserved up front by
its own allocator, or a frame loop that cannot afford the device-wide
synchronisation cudaMalloc and cudaFree may cause) get an entry point whose
scratch lives in one fixed static device array.  Through the C ABI, two calls
in a row must give the same image, per-pixel counts and stats as
ctf_filter_host on the same arguments (counts and stats exactly, pixels within
1e-6 relative, the tolerance of the other parity tests), and a view too large
for the array must be refused.  For learned textures as well as block
textures the library's own allocation counter must not move during the calls,
and in a fresh process (where no earlier call has set up anything lazily) the
first calls must leave the device's free memory unchanged.  This file is
collected last so that a run that stops at the first failure has already run
every other test."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2506_17770_gb300 import _ctf, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def setup():
    from paper_2506_17770_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    Wt = Ht = 2048
    tex = _ctf.ctf_texture_create(Wt, Ht, synth.random_blocks(Wt, Ht))
    sc = synth.ground_plane_with_quads(1024, 768, Wt, Ht)
    yield tex, sc
    _ctf.ctf_texture_destroy(tex)


def _host(sc):
    H, W = sc.H, sc.W
    return (torch.from_numpy(sc.uv).pin_memory(), torch.from_numpy(sc.jac).pin_memory(),
            torch.from_numpy(sc.coverage).pin_memory(),
            torch.empty((H, W, 4), dtype=torch.float32).pin_memory(),
            torch.empty((H, W), dtype=torch.uint8).pin_memory())


def test_noalloc_matches_host_entry_point_on_two_calls_in_a_row(setup):
    tex, sc = setup
    W, H = sc.W, sc.H
    uv, jac, cov, out, ev = _host(sc)
    _, _, _, out_ref, ev_ref = _host(sc)
    for alg, seed, opts in (("mask", 0, {"mask_dim": 11}), ("box", 12345, None)):
        out.fill_(-1.0)
        ev.fill_(77)
        st = _ctf.ctf_filter_host_noalloc(tex, uv, jac, cov, W, H, 0, alg, seed, opts, out, ev, stats=True)
        st_ref = _ctf.ctf_filter_host(tex, uv, jac, cov, W, H, 0, alg, seed, opts, out_ref, ev_ref, stats=True)
        assert st == st_ref
        assert st["pixels_active"] == W * H and st["tiles_success"] > 0
        np.testing.assert_array_equal(ev.numpy(), ev_ref.numpy())
        np.testing.assert_allclose(out.numpy(), out_ref.numpy(), rtol=1e-6, atol=1e-7)


def _learned_texture(Wt, Ht, seed=4):
    g = np.random.default_rng(seed)
    lat = [g.normal(0, 1.0, (Ht // 4, Wt // 4, 8)).astype(np.float32),
           g.normal(0, 1.0, (Ht // 8, Wt // 8, 8)).astype(np.float32)]
    p = (g.normal(0, 0.35, (64, 16)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
         g.normal(0, 0.18, (64, 64)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
         g.normal(0, 0.04, (4, 64)).astype(np.float32), np.array([0.5, 0.5, 0.5, 0.9], np.float32))
    return _ctf.ctf_texture_create_mlp(Wt, Ht, _ctf.CTF_EVAL_MLP_FP16, lat, *p)


def test_noalloc_learned_texture_allocates_nothing_and_matches(setup):
    """A learned (FP16 MLP) texture: the path that reports a wait that gave up
    through the library's error word, which must not need an allocation."""
    _, sc = setup
    W, H = sc.W, sc.H
    ltex = _learned_texture(2048, 2048)
    try:
        uv, jac, cov, out, ev = _host(sc)
        _, _, _, out_ref, ev_ref = _host(sc)
        for alg, seed, opts in (("mask", 0, {"mask_dim": 11}), ("box", 99, None), ("mask", 5, {"mask_dim": 11})):
            out.fill_(-1.0)
            ev.fill_(77)
            torch.cuda.synchronize()
            c0 = _ctf.ctf_debug_device_allocations()
            st = _ctf.ctf_filter_host_noalloc(ltex, uv, jac, cov, W, H, 0, alg, seed, opts, out, ev, stats=True)
            assert _ctf.ctf_debug_device_allocations() == c0
            _ctf.ctf_sync_check()
            st_ref = _ctf.ctf_filter_host(ltex, uv, jac, cov, W, H, 0, alg, seed, opts, out_ref, ev_ref, stats=True)
            assert st == st_ref
            assert st["tiles_success"] > 0
            np.testing.assert_array_equal(ev.numpy(), ev_ref.numpy())
            np.testing.assert_allclose(out.numpy(), out_ref.numpy(), rtol=1e-6, atol=1e-7)
    finally:
        _ctf.ctf_texture_destroy(ltex)


_FRESH = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2506_17770_gb300 import _ctf, synth
torch.cuda.set_device(0)
Wt = Ht = 1024
btex = _ctf.ctf_texture_create(Wt, Ht, synth.random_blocks(Wt, Ht))
g = np.random.default_rng(4)
lat = [g.normal(0, 1.0, (Ht // 4, Wt // 4, 8)).astype(np.float32),
       g.normal(0, 1.0, (Ht // 8, Wt // 8, 8)).astype(np.float32)]
p = (g.normal(0, 0.35, (64, 16)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
     g.normal(0, 0.18, (64, 64)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
     g.normal(0, 0.04, (4, 64)).astype(np.float32), np.array([0.5, 0.5, 0.5, 0.9], np.float32))
ltex = _ctf.ctf_texture_create_mlp(Wt, Ht, _ctf.CTF_EVAL_MLP_FP16, lat, *p)
sc = synth.perspective_view(320, 200, Wt, Ht, 1.0, 12.0, seed=7)
H, W = 200, 320
uv = torch.from_numpy(sc.uv).pin_memory()
jac = torch.from_numpy(sc.jac).pin_memory()
outs = [torch.empty((H, W, 4)).pin_memory() for _ in range(4)]
evs = [torch.empty((H, W), dtype=torch.uint8).pin_memory() for _ in range(4)]
# load and run the kernels once through the device entry point, which
# allocates nothing without stats either, so no first launch lands below
d_out = torch.empty((H, W, 4), device="cuda")
d_ev = torch.empty((H, W), dtype=torch.uint8, device="cuda")
c_warm = _ctf.ctf_debug_device_allocations()
for tex in (ltex, btex):
    _ctf.ctf_filter(tex, uv.cuda(), jac.cuda(), None, W, H, 0, "mask", 1, {"mask_dim": 11}, d_out, d_ev)
torch.cuda.synchronize()
res = {"warm_allocs": _ctf.ctf_debug_device_allocations() - c_warm}
c0 = _ctf.ctf_debug_device_allocations()
free0 = torch.cuda.mem_get_info()[0]
stats = []
for i, tex in enumerate((ltex, ltex, btex, btex)):
    stats.append(_ctf.ctf_filter_host_noalloc(tex, uv, jac, None, W, H, 0, "mask", 1, {"mask_dim": 11},
                                              outs[i], evs[i], stats=True))
_ctf.ctf_sync_check()
torch.cuda.synchronize()
res["allocs"] = _ctf.ctf_debug_device_allocations() - c0
res["free_before"] = free0
res["free_after"] = torch.cuda.mem_get_info()[0]
# the same views through the allocating host entry point, afterwards
ref_out = torch.empty((H, W, 4)).pin_memory()
ref_ev = torch.empty((H, W), dtype=torch.uint8).pin_memory()
ok = []
for i, tex in enumerate((ltex, ltex, btex, btex)):
    st = _ctf.ctf_filter_host(tex, uv, jac, None, W, H, 0, "mask", 1, {"mask_dim": 11}, ref_out, ref_ev, stats=True)
    ok.append(bool(st == stats[i] and torch.equal(ref_ev, evs[i]) and
                   np.allclose(outs[i].numpy(), ref_out.numpy(), rtol=1e-6, atol=1e-7)))
res["match"] = ok
print("RESULT " + json.dumps(res))
"""


def test_noalloc_first_calls_in_a_fresh_process_leave_device_memory_alone():
    """Nothing set up lazily by earlier calls: the first no-allocation calls
    of a process, on a learned and a block texture, must neither reach the
    library's allocation routine nor change the device's free memory.  Module
    loading is made eager so that loading the library's code and static data
    (the scratch array itself) happens before the measurement."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", _FRESH, root],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert res["warm_allocs"] == 0, res
    assert res["allocs"] == 0, res
    assert res["free_after"] == res["free_before"], res
    assert all(res["match"]), res


def test_noalloc_refuses_a_view_larger_than_its_array(setup):
    tex, _ = setup
    W, H = 1920, 1080
    uv = torch.zeros((H, W, 2)).pin_memory()
    jac = torch.zeros((H, W, 4)).pin_memory()
    out = torch.zeros((H, W, 4)).pin_memory()
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_filter_host_noalloc(tex, uv, jac, None, W, H, 0, "box", 0, None, out, None)
    assert ei.value.status == _ctf.CTF_ERR_ARG
    assert "scratch" in str(ei.value)
