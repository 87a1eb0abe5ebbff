"""ctf_filter_host_noalloc: the host-buffer filter for callers that cannot let
the library allocate device memory.

Such callers (a renderer or plug-in whose video memory is reserved up front by
its own allocator, or a frame loop that cannot afford the device-wide
synchronisation cudaMalloc and cudaFree may cause) get an entry point whose
scratch lives in one fixed static device array.  Through the C ABI, two calls
in a row must give the same image, per-pixel counts and stats as
ctf_filter_host on the same arguments (counts and stats exactly, pixels within
1e-6 relative, the tolerance of the other parity tests), and a view too large
for the array must be refused.  This file is collected last so that a run that
stops at the first failure has already run every other test."""
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
