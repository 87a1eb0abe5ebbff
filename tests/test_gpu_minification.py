"""The minification vote (step a2) on the GPU: the hand-derived cases of the
oracle's pins, run through the C ABI on both decoders.

Each case is one tile whose pixels all sample one point (a 2x2 footprint)
and whose lane 17 (or a chosen lane) carries the Jacobian under test; the
tile succeeds (4 texels, counted once each) unless the vote sends it to
one-tap STF (every active pixel counts 1).  The expected outcome is the
flag written by hand in the pin file; the exact-decode images and counts
must also equal the oracle's bit for bit, and the learned-decode counts the
oracle's."""
import numpy as np
import pytest

import oracle
from paper_2506_17770_gb300 import _ctf, synth

import test_oracle_minification_pins as pins

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ALG_NAMES = {2: "list_merge", 3: "box", 4: "mask"}


@pytest.fixture(scope="module")
def textures():
    from paper_2506_17770_gb300 import build
    build.build()
    oracle.build()
    blocks = synth.random_blocks(pins.WT, pins.HT)
    tex = _ctf.ctf_texture_create(pins.WT, pins.HT, blocks)
    g = np.random.default_rng(9)
    lat = [g.normal(0, 1.0, (pins.HT // 4, pins.WT // 4, 8)).astype(np.float32),
           g.normal(0, 1.0, (pins.HT // 8, pins.WT // 8, 8)).astype(np.float32)]
    p = (g.normal(0, 0.35, (64, 16)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
         g.normal(0, 0.18, (64, 64)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
         g.normal(0, 0.04, (4, 64)).astype(np.float32), np.array([0.5, 0.5, 0.5, 0.9], np.float32))
    ltex = _ctf.ctf_texture_create_mlp(pins.WT, pins.HT, _ctf.CTF_EVAL_MLP_FP16, lat, *p)
    yield blocks, tex, ltex
    _ctf.ctf_texture_destroy(tex)
    _ctf.ctf_texture_destroy(ltex)


def _gpu(tex, uv, jac, cov, alg, tile_w, tile_h):
    H, W = uv.shape[:2]
    out = torch.full((H, W, 4), -3.0, device="cuda")
    ev = torch.full((H, W), 99, dtype=torch.uint8, device="cuda")
    c = None if cov is None else torch.from_numpy(cov).cuda()
    st = _ctf.ctf_filter(tex, torch.from_numpy(uv).cuda(), torch.from_numpy(jac).cuda(), c, W, H, 0,
                         ALG_NAMES[alg], 0, {"tile_w": tile_w, "tile_h": tile_h}, out, ev, stats=True)
    _ctf.ctf_sync_check()
    return out.cpu().numpy(), ev.cpu().numpy(), st


def _check(textures, T, alg, minified, lane=17, inactive=False, tile_w=8, tile_h=4):
    blocks, tex, ltex = textures
    uv, jac, cov = pins._frame(T, lane, inactive, tile_w, tile_h)
    ref, ref_ev, ref_st = oracle.filter_frame(blocks, pins.WT, pins.HT, uv, jac, cov, alg=alg, tile_w=tile_w,
                                              tile_h=tile_h)
    for t in (tex, ltex):
        out, ev, st = _gpu(t, uv, jac, cov, alg, tile_w, tile_h)
        assert st["tiles_fallback_minified"] == (1 if minified else 0)
        assert st["tiles_success"] == (0 if minified else 1)
        np.testing.assert_array_equal(ev, ref_ev)
        assert st["texel_evals"] == ref_st["texel_evals"]
        if minified:
            assert np.all(ev[cov != 0] == 1) if cov is not None else np.all(ev == 1)
        else:
            assert int(ev.sum()) == 4
        if t is tex:
            assert st == ref_st
            assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("alg", [2, 3, 4])
@pytest.mark.parametrize("name,T,minified", pins.CASES, ids=[c[0] for c in pins.CASES])
def test_minification_flag_on_the_gpu(textures, alg, name, T, minified):
    _check(textures, T, alg, minified)


@pytest.mark.parametrize("lane", [0, 31])
def test_one_minified_lane_and_an_inactive_one(textures, lane):
    _check(textures, (2.0, 0.0, 0.0, 0.0), 4, True, lane=lane)
    _check(textures, (2.0, 0.0, 0.0, 0.0), 4, False, lane=lane, inactive=True)


@pytest.mark.parametrize("shape", [(4, 8), (16, 2)])
def test_vote_with_other_tile_shapes_on_the_gpu(textures, shape):
    tw, th = shape
    _check(textures, (0.0, 0.0, 0.0, 1.5), 4, True, lane=31, tile_w=tw, tile_h=th)
    _check(textures, (0.0, 0.0, 0.0, 1.0), 4, False, lane=31, tile_w=tw, tile_h=th)
