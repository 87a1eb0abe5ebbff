"""GPU parity of the exact-decode path against the CPU oracle, through the C ABI.

Bar: per-pixel texel-evaluation counts and per-tile outcomes bit-exact; FP32
pixels within 1e-6 relative (the selection and weight arithmetic is the same
sequence of IEEE operations on both sides, so the pixels are also checked
for bit equality separately)."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_17770_gb300 import _ctf, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

RTOL = 1e-6
ALGS = {"4tap": 0, "stf": 1, "list_merge": 2, "box": 3, "mask": 4}
TILES = [(8, 4), (4, 8), (16, 2)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_17770_gb300 import build
    build.build()
    oracle.build()


class Tex:
    def __init__(self, blocks, Wt, Ht):
        self.blocks, self.Wt, self.Ht = blocks, Wt, Ht
        self.h = _ctf.ctf_texture_create(Wt, Ht, np.ascontiguousarray(blocks))

    def close(self):
        _ctf.ctf_texture_destroy(self.h)


def gpu_filter(tex, scene_uv, scene_jac, cov, alg, seed=0, view=0, opts=None, stats=True):
    H, W = scene_uv.shape[:2]
    uv = torch.from_numpy(np.ascontiguousarray(scene_uv)).cuda()
    jac = torch.from_numpy(np.ascontiguousarray(scene_jac)).cuda()
    c = None if cov is None else torch.from_numpy(np.ascontiguousarray(cov)).cuda()
    out = torch.full((H, W, 4), -7.0, dtype=torch.float32, device="cuda")
    ev = torch.full((H, W), 99, dtype=torch.uint8, device="cuda")
    st = _ctf.ctf_filter(tex.h, uv, jac, c, W, H, view, alg, seed, opts, out, ev, stats=stats)
    torch.cuda.synchronize()
    return out.cpu().numpy(), ev.cpu().numpy(), st


def cpu_filter(tex, uv, jac, cov, alg, seed=0, view=0, opts=None):
    o = {"tile_w": 8, "tile_h": 4, "budget": 32, "mask_dim": 16, "edge_remap": 1}
    o.update(opts or {})
    return oracle.filter_frame(tex.blocks, tex.Wt, tex.Ht, uv, jac, cov, view=view, alg=ALGS[alg], seed=seed, **o)


def assert_parity(g, c, bit_exact=True):
    gout, gev, gst = g
    cout, cev, cst = c
    np.testing.assert_array_equal(gev, cev)
    assert gst == cst
    np.testing.assert_allclose(gout, cout, rtol=RTOL, atol=1e-7)
    if bit_exact:
        assert np.array_equal(gout.view(np.uint32), cout.view(np.uint32))


# ---------------------------------------------------------------------------
# Small magnified plane: 128x128 frame, 64x64 texture, uniform 4x magnification
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small():
    Wt = Ht = 64
    tex = Tex(synth.random_blocks(Wt, Ht), Wt, Ht)
    sc = synth.magnified_plane(128, 128, Wt, Ht, scale=0.25)
    yield tex, sc
    tex.close()


@pytest.mark.parametrize("alg", list(ALGS))
@pytest.mark.parametrize("tile", TILES)
def test_small_plane_all_algorithms(small, alg, tile):
    tex, sc = small
    opts = {"tile_w": tile[0], "tile_h": tile[1]}
    g = gpu_filter(tex, sc.uv, sc.jac, None, alg, opts=opts)
    c = cpu_filter(tex, sc.uv, sc.jac, None, alg, opts=opts)
    assert_parity(g, c)
    if alg in ("box", "mask", "list_merge") and tile == (8, 4):
        # every warp is magnified 4x: all succeed, well under one evaluation per pixel
        assert g[2]["tiles_success"] == g[2]["tiles_total"]
        assert g[2]["texel_evals"] / g[2]["pixels_active"] < 0.75


def test_success_equals_4tap_bitwise(small):
    tex, sc = small
    ref = gpu_filter(tex, sc.uv, sc.jac, None, "4tap")[0]
    for alg in ("box", "mask", "list_merge"):
        out = gpu_filter(tex, sc.uv, sc.jac, None, alg)[0]
        assert np.array_equal(out.view(np.uint32), ref.view(np.uint32)), alg


# ---------------------------------------------------------------------------
# Full frame: 1920x1080, 2048^2 texture, perspective ground plane + quads
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def frame():
    Wt = Ht = 2048
    tex = Tex(synth.random_blocks(Wt, Ht), Wt, Ht)
    sc = synth.ground_plane_with_quads(1920, 1080, Wt, Ht)
    yield tex, sc
    tex.close()


@pytest.mark.parametrize("alg", list(ALGS))
def test_full_frame_parity(frame, alg):
    tex, sc = frame
    g = gpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, seed=0)
    c = cpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, seed=0)
    assert_parity(g, c)
    if alg in ("box", "mask", "list_merge"):
        st = g[2]
        assert st["tiles_success"] > 0 and st["tiles_fallback_minified"] > 0 and st["tiles_fallback_budget"] > 0


@pytest.mark.parametrize("tile", [(4, 8), (16, 2)])
@pytest.mark.parametrize("alg", ["box", "mask"])
def test_full_frame_other_tiles(frame, alg, tile):
    tex, sc = frame
    opts = {"tile_w": tile[0], "tile_h": tile[1]}
    assert_parity(gpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, seed=5, opts=opts),
                  cpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, seed=5, opts=opts))


def test_full_frame_mask11_and_seed_view(frame):
    tex, sc = frame
    opts = {"mask_dim": 11}
    assert_parity(gpu_filter(tex, sc.uv, sc.jac, sc.coverage, "mask", seed=2**63 + 12345, view=9, opts=opts),
                  cpu_filter(tex, sc.uv, sc.jac, sc.coverage, "mask", seed=2**63 + 12345, view=9, opts=opts))


# ---------------------------------------------------------------------------
# Ragged frames, coverage holes, options, degenerate inputs
# ---------------------------------------------------------------------------
def _mixed_scene(W, H, seed):
    g = np.random.default_rng(seed)
    uv = np.zeros((H, W, 2))
    jac = np.zeros((H, W, 4))
    for ty in range(0, H, 4):
        for tx in range(0, W, 8):
            m = math.exp(g.uniform(math.log(0.6), math.log(8.0)))
            r = g.uniform(0, 2 * math.pi)
            c, s = math.cos(r), math.sin(r)
            o = g.uniform(-3, 60, 2)  # some tiles hang over the texture edge (clamping)
            ly, lx = np.meshgrid(np.arange(4) + 0.5, np.arange(8) + 0.5, indexing="ij")
            X = (c * lx - s * ly) / m + o[0]
            Y = (s * lx + c * ly) / m + o[1]
            hh, ww = min(4, H - ty), min(8, W - tx)
            sl = (slice(ty, ty + hh), slice(tx, tx + ww))
            uv[sl + (0,)] = (X / 64)[:hh, :ww]
            uv[sl + (1,)] = (Y / 64)[:hh, :ww]
            jac[sl] = np.array([c / m / 64, s / m / 64, -s / m / 64, c / m / 64])
    cov = (g.uniform(size=(H, W)) > 0.2).astype(np.uint8)
    uv = uv.astype(np.float32)
    uv[0, 0] = np.nan
    uv[H // 2, W // 3] = [3e7, 0.5]
    jac = jac.astype(np.float32)
    jac[H - 1, W - 1] = np.inf
    return uv, jac, cov


@pytest.fixture(scope="module")
def mixed():
    tex = Tex(synth.random_blocks(64, 64, seed=7), 64, 64)
    yield tex
    tex.close()


@pytest.mark.parametrize("W,H", [(133, 77), (8, 4), (1, 1), (17, 3), (250, 131)])
@pytest.mark.parametrize("alg", list(ALGS))
def test_ragged_mixed(mixed, W, H, alg):
    uv, jac, cov = _mixed_scene(W, H, seed=W * 1000 + H)
    for opts in (None, {"edge_remap": 0}, {"budget": 9, "mask_dim": 11}, {"tile_w": 16, "tile_h": 2, "budget": 20}):
        assert_parity(gpu_filter(mixed, uv, jac, cov, alg, seed=77, opts=opts),
                      cpu_filter(mixed, uv, jac, cov, alg, seed=77, opts=opts))


@pytest.mark.parametrize("fallback", [1, 2])
@pytest.mark.parametrize("alg", ["box", "mask", "list_merge"])
def test_fallback_c_and_cplus(frame, mixed, alg, fallback):
    """Fallbacks C (1) and C+ (2) of Sec. 3.4 in place of one-tap STF on the
    over-budget tiles: the full view, and ragged frames with coverage holes,
    clamped edges and the option sets of the ragged test."""
    tex, sc = frame
    for opts in ({"fallback": fallback}, {"fallback": fallback, "mask_dim": 11, "tile_w": 4, "tile_h": 8}):
        g = gpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, seed=31, opts=opts)
        assert_parity(g, cpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, seed=31, opts=opts))
        assert g[2]["tiles_fallback_budget"] > 0
    for W, H in ((133, 77), (17, 3), (250, 131)):
        uv, jac, cov = _mixed_scene(W, H, seed=W * 1000 + H)
        for opts in ({"fallback": fallback}, {"fallback": fallback, "edge_remap": 0},
                     {"fallback": fallback, "budget": 9, "mask_dim": 11},
                     {"fallback": fallback, "tile_w": 16, "tile_h": 2, "budget": 20}):
            assert_parity(gpu_filter(mixed, uv, jac, cov, alg, seed=77, opts=opts),
                          cpu_filter(mixed, uv, jac, cov, alg, seed=77, opts=opts))


@pytest.mark.parametrize("alg", ["box", "mask", "list_merge"])
def test_two_texels_per_lane(frame, mixed, alg):
    """Up to two texels per lane (budget up to 64), alone and with fallback
    C+, on the full view, on ragged frames with the option sets of the
    ragged test, and on rotated head-on quads just above magnification 1,
    where every 8x4 wave succeeds (Sec. 5)."""
    tex, sc = frame
    for opts in ({"texels_per_lane": 2, "budget": 64}, {"texels_per_lane": 2, "budget": 64, "mask_dim": 11},
                 {"texels_per_lane": 2, "budget": 40, "fallback": 2}):
        g = gpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, seed=3, opts=opts)
        assert_parity(g, cpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, seed=3, opts=opts))
    for W, H in ((133, 77), (17, 3), (250, 131)):
        uv, jac, cov = _mixed_scene(W, H, seed=W * 1000 + H)
        for opts in ({"texels_per_lane": 2, "budget": 64}, {"texels_per_lane": 2, "budget": 64, "edge_remap": 0},
                     {"texels_per_lane": 2, "budget": 48, "mask_dim": 11},
                     {"texels_per_lane": 2, "budget": 64, "tile_w": 16, "tile_h": 2, "fallback": 1}):
            assert_parity(gpu_filter(mixed, uv, jac, cov, alg, seed=77, opts=opts),
                          cpu_filter(mixed, uv, jac, cov, alg, seed=77, opts=opts))
    q = synth.rotated_quad_tiles(1.001, np.arange(0, 91, 3.0), 40)
    qt = Tex(synth.random_blocks(4096, 4096, seed=16), 4096, 4096)
    try:
        opts = {"texels_per_lane": 2, "budget": 64}
        g = gpu_filter(qt, q.uv, q.jac, None, alg, opts=opts)
        assert_parity(g, cpu_filter(qt, q.uv, q.jac, None, alg, opts=opts))
        if alg != "box":
            assert g[2]["tiles_success"] == g[2]["tiles_total"]
    finally:
        qt.close()


@pytest.mark.parametrize("flt", [1, 2])
@pytest.mark.parametrize("alg", list(ALGS))
def test_bicubic_filters(frame, mixed, alg, flt):
    """The bicubic filters of Sec. 4.2 (1 cubic B-spline, 2 Catmull-Rom) for
    every algorithm: the full view, and ragged frames with coverage holes,
    clamped edges and the option sets of the ragged test."""
    tex, sc = frame
    for opts in ({"filter": flt}, {"filter": flt, "mask_dim": 11, "tile_w": 4, "tile_h": 8}):
        g = gpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, seed=11, opts=opts)
        assert_parity(g, cpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, seed=11, opts=opts))
        if alg in ("box", "mask", "list_merge"):
            assert g[2]["tiles_success"] > 0
    for W, H in ((133, 77), (17, 3), (250, 131)):
        uv, jac, cov = _mixed_scene(W, H, seed=W * 1000 + H)
        for opts in ({"filter": flt}, {"filter": flt, "edge_remap": 0}, {"filter": flt, "budget": 20, "mask_dim": 11},
                     {"filter": flt, "tile_w": 16, "tile_h": 2}):
            assert_parity(gpu_filter(mixed, uv, jac, cov, alg, seed=77, opts=opts),
                          cpu_filter(mixed, uv, jac, cov, alg, seed=77, opts=opts))


def test_empty_and_uncovered(mixed):
    uv, jac, cov = _mixed_scene(40, 20, seed=1)
    z = np.zeros((20, 40), np.uint8)
    g = gpu_filter(mixed, uv, jac, z, "mask")
    assert np.all(g[0] == 0) and np.all(g[1] == 0) and g[2]["tiles_empty"] == g[2]["tiles_total"]
    # zero-sized frame: a no-op that still reports zero stats
    out = torch.zeros(0, device="cuda")
    st = _ctf.ctf_filter(mixed.h, out, out, None, 0, 5, 0, "box", 0, None, out, None, stats=True)
    assert st["tiles_total"] == 0


def test_fig4_thresholds_on_gpu(built):
    """The magnification thresholds of Fig. 4 hold on the GPU path too (8x4
    waves, every rotation 0..90 degrees): all warps succeed just above 1.59
    (List Merge, Mask) and 2.35 (Box), and the per-tile outcome matches the
    oracle below them."""
    blocks = synth.random_blocks(4096, 4096, seed=16)
    tex = Tex(blocks, 4096, 4096)
    try:
        for m, alg in ((1.60, "mask"), (1.60, "list_merge"), (2.36, "box"), (1.55, "mask"), (2.30, "box")):
            sc = synth.rotated_quad_tiles(m, np.arange(0, 91, 1.0), 80)
            g = gpu_filter(tex, sc.uv, sc.jac, None, alg)
            c = cpu_filter(tex, sc.uv, sc.jac, None, alg)
            assert_parity(g, c)
            if m in (1.60, 2.36):
                assert g[2]["tiles_success"] == g[2]["tiles_total"], (m, alg)
            else:
                assert g[2]["tiles_fallback_budget"] > 0, (m, alg)
    finally:
        tex.close()


@pytest.mark.parametrize("alg,opts", [("4tap", None), ("stf", None), ("box", None), ("mask", {"mask_dim": 11}),
                                      ("list_merge", {"tile_w": 4, "tile_h": 8}), ("mask", {"fallback": 2}),
                                      ("mask", {"texels_per_lane": 2, "budget": 64}),
                                      ("mask", {"filter": 2}), ("box", {"tile_w": 16, "tile_h": 2, "filter": 1})])
def test_host_entry_point_matches_device(frame, alg, opts):
    """ctf_filter_host on page-locked buffers filters them in place (the
    kernel reads the inputs and writes the image in host memory; the counts
    come back in one copy, into page-locked or pageable memory); on pageable
    buffers it stages them in 4 row bands of a view of more than 2^20
    pixels, whose copies overlap the filtering of their neighbours, each band
    filtered as the part of the view it is.  Either way the image and counts
    equal one ctf_filter call on the whole view (the STF draws of minified
    and over-budget tiles included)."""
    tex, sc = frame
    H, W = sc.H, sc.W
    assert W * H >= 1 << 20
    g = gpu_filter(tex, sc.uv, sc.jac, sc.coverage, alg, opts=opts, seed=3)
    assert g[2]["tiles_fallback_minified"] + g[2]["tiles_direct"] > 0
    for pinned, ev_pinned in ((True, True), (True, False), (False, False)):
        def host(a, pin=pinned):
            t = torch.from_numpy(np.ascontiguousarray(a))
            return t.pin_memory() if pin else t.clone()
        uv, jac, cov = host(sc.uv), host(sc.jac), host(sc.coverage)
        out = host(np.zeros((H, W, 4), np.float32))
        ev = host(np.full((H, W), 77, np.uint8), ev_pinned)
        st = _ctf.ctf_filter_host(tex.h, uv, jac, cov, W, H, 0, alg, 3, opts, out, ev, stats=True)
        assert st == g[2], pinned
        assert np.array_equal(out.numpy().view(np.uint32), g[0].view(np.uint32)), pinned
        assert np.array_equal(ev.numpy(), g[1]), pinned


def test_argument_errors(mixed):
    uv = torch.zeros((4, 8, 2), device="cuda")
    jac = torch.zeros((4, 8, 4), device="cuda")
    out = torch.zeros((4, 8, 4), device="cuda")
    bad = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_filter(mixed.h, uv, bad.data_ptr() + 4, None, 8, 4, 0, "box", 0, None, out, None)
    assert ei.value.status == _ctf.CTF_ERR_ALIGN
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_filter(mixed.h, uv, jac, None, 8, 4, 0, "box", 0, {"tile_w": 4, "tile_h": 4}, out, None)
    assert ei.value.status == _ctf.CTF_ERR_ARG
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_filter(mixed.h, uv, jac, None, 8, 4, 0, 9, 0, None, out, None)
    assert ei.value.status == _ctf.CTF_ERR_ARG
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_filter(mixed.h, uv, jac, None, 40000, 4, 0, "box", 0, None, out, None)
    assert ei.value.status == _ctf.CTF_ERR_ARG
