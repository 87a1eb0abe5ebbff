"""Batched persistent launch: every view of a mixed batch (block and learned
textures, uneven and ragged sizes, coverage holes) must come out bit-identical
to ctf_filter on that view alone, with summed stats; the captured graph must
replay the same result; the autotuner must return a configuration whose
results again equal the per-view calls.  Exact views are also checked against
the CPU oracle directly."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_17770_gb300 import _ctf, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_17770_gb300 import build
    build.build()
    oracle.build()


def _learned_params(seed, Wt, Ht):
    g = np.random.default_rng(seed)
    lat = [g.normal(0, 1.0, (Ht // 4, Wt // 4, 8)).astype(np.float32),
           g.normal(0, 1.0, (Ht // 8, Wt // 8, 8)).astype(np.float32)]
    return lat, (g.normal(0, 0.35, (64, 16)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
                 g.normal(0, 0.18, (64, 64)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
                 g.normal(0, 0.04, (4, 64)).astype(np.float32), np.array([0.5, 0.5, 0.5, 0.9], np.float32))


@pytest.fixture(scope="module")
def textures():
    blocks = synth.random_blocks(256, 256, seed=31)
    tb = _ctf.ctf_texture_create(256, 256, blocks)
    lat, p = _learned_params(5, 128, 128)
    tl = _ctf.ctf_texture_create_mlp(128, 128, _ctf.CTF_EVAL_MLP_FP16, lat, *p)
    lat2, p2 = _learned_params(6, 64, 64)
    tl2 = _ctf.ctf_texture_create_mlp(64, 64, _ctf.CTF_EVAL_MLP_FP16, lat2, *p2)
    yield {"block": (tb, blocks, 256), "learned": (tl, None, 128), "learned2": (tl2, None, 64)}
    for t in (tb, tl, tl2):
        _ctf.ctf_texture_destroy(t)


def _make_views(textures, n=9, seed=3):
    g = np.random.default_rng(seed)
    kinds = ["block", "learned", "block", "learned2"]
    views = []
    for i in range(n):
        kind = kinds[i % len(kinds)]
        tex, blocks, dim = textures[kind]
        W, H = int(g.integers(1, 300)), int(g.integers(1, 200))
        if i == 0:
            W, H = 0, 7  # an empty view
        lo, hi = sorted(np.exp(g.uniform(math.log(0.5), math.log(12.0), 2)))
        sc = synth.perspective_view(max(W, 1), max(H, 1), dim, dim, float(lo), float(hi), seed=seed, view=i)
        uv, jac, cov = sc.uv[:H, :W], sc.jac[:H, :W], sc.coverage[:H, :W]
        cov = cov & (g.uniform(size=cov.shape) > 0.05).astype(np.uint8)
        v = {"tex": tex, "kind": kind, "blocks": blocks, "dim": dim, "width": W, "height": H, "view_id": 100 + i,
             "np_uv": np.ascontiguousarray(uv), "np_jac": np.ascontiguousarray(jac), "np_cov": np.ascontiguousarray(cov),
             "uv": torch.from_numpy(np.ascontiguousarray(uv)).cuda(),
             "jac": torch.from_numpy(np.ascontiguousarray(jac)).cuda(),
             "coverage": torch.from_numpy(np.ascontiguousarray(cov)).cuda(),
             "out_rgba": torch.full((max(H, 1), max(W, 1), 4), -5.0, device="cuda"),
             "out_evals": torch.full((max(H, 1), max(W, 1)), 99, dtype=torch.uint8, device="cuda")}
        views.append(v)
    return views


def _single(v, alg, seed, fopts):
    out = torch.full_like(v["out_rgba"], -5.0)
    ev = torch.full_like(v["out_evals"], 99)
    st = _ctf.ctf_filter(v["tex"], v["uv"], v["jac"], v["coverage"], v["width"], v["height"], v["view_id"], alg,
                         seed, fopts, out, ev, stats=True)
    return out.cpu().numpy(), ev.cpu().numpy(), st


def _sum_stats(stats):
    tot = {}
    for s in stats:
        for k, val in s.items():
            tot[k] = tot.get(k, 0) + val
    return tot


@pytest.mark.parametrize("alg", ["4tap", "stf", "list_merge", "box", "mask"])
def test_batch_equals_per_view_calls(textures, alg):
    views = _make_views(textures)
    o = _ctf.batch_opts(tile_w=8, tile_h=4, mask_dim=11 if alg == "mask" else 16, items_per_fetch=2, ctas_per_sm=4)
    fopts = {"tile_w": 8, "tile_h": 4, "mask_dim": o.filter.mask_dim}
    st = _ctf.ctf_filter_batch(views, alg, 12345, o, stats=True)
    _ctf.ctf_sync_check()
    singles = []
    for v in views:
        ref, ref_ev, ref_st = _single(v, alg, 12345, fopts)
        singles.append(ref_st)
        got, got_ev = v["out_rgba"].cpu().numpy(), v["out_evals"].cpu().numpy()
        H, W = v["height"], v["width"]
        assert np.array_equal(got[:H, :W].view(np.uint32), ref[:H, :W].view(np.uint32)), (alg, v["kind"], W, H)
        assert np.array_equal(got_ev[:H, :W], ref_ev[:H, :W])
    assert st == _sum_stats(singles)


def test_batch_exact_views_match_oracle(textures):
    views = _make_views(textures, n=6, seed=8)
    o = _ctf.batch_opts(tile_w=4, tile_h=8, items_per_fetch=1, ctas_per_sm=2)
    _ctf.ctf_filter_batch(views, "box", 7, o)
    _ctf.ctf_sync_check()
    for v in views:
        if v["kind"] != "block" or v["width"] == 0:
            continue
        ref, ref_ev, _ = oracle.filter_frame(v["blocks"], v["dim"], v["dim"], v["np_uv"], v["np_jac"], v["np_cov"],
                                             view=v["view_id"], alg=oracle.ALG_BOX, seed=7, tile_w=4, tile_h=8)
        H, W = v["height"], v["width"]
        np.testing.assert_array_equal(v["out_evals"].cpu().numpy()[:H, :W], ref_ev)
        assert np.array_equal(v["out_rgba"].cpu().numpy()[:H, :W].view(np.uint32), ref.view(np.uint32))


def test_graph_replays_the_batch(textures):
    views = _make_views(textures, n=7, seed=11)
    o = _ctf.batch_opts(items_per_fetch=4, ctas_per_sm=4)
    _ctf.ctf_filter_batch(views, "mask", 3, o)
    _ctf.ctf_sync_check()
    first = [(v["out_rgba"].cpu().numpy().copy(), v["out_evals"].cpu().numpy().copy()) for v in views]
    for v in views:
        v["out_rgba"].fill_(-1.0)
        v["out_evals"].fill_(7)
    g = _ctf.ctf_batch_graph_create(views, "mask", 3, o)
    try:
        for _ in range(3):
            _ctf.ctf_batch_graph_launch(g)
        _ctf.ctf_sync_check()
    finally:
        _ctf.ctf_batch_graph_destroy(g)
    for v, (a, e) in zip(views, first):
        H, W = v["height"], v["width"]
        assert np.array_equal(v["out_rgba"].cpu().numpy()[:H, :W].view(np.uint32), a[:H, :W].view(np.uint32))
        assert np.array_equal(v["out_evals"].cpu().numpy()[:H, :W], e[:H, :W])


def test_autotune_picks_a_consistent_configuration(textures):
    views = _make_views(textures, n=5, seed=13)
    best, ms = _ctf.ctf_batch_autotune(views, "box", 1)
    d = best.as_dict()
    assert (d["tile_w"], d["tile_h"]) in ((8, 4), (4, 8), (16, 2))
    assert d["items_per_fetch"] in (1, 2, 4, 8) and d["ctas_per_sm"] in (2, 4) and ms > 0
    assert d["solo_tiles"] in (0, 4096, 16384, 65536)
    _ctf.ctf_filter_batch(views, "box", 1, best)
    _ctf.ctf_sync_check()
    fopts = {"tile_w": d["tile_w"], "tile_h": d["tile_h"]}
    for v in views:
        ref, ref_ev, _ = _single(v, "box", 1, fopts)
        H, W = v["height"], v["width"]
        assert np.array_equal(v["out_rgba"].cpu().numpy()[:H, :W].view(np.uint32), ref[:H, :W].view(np.uint32))


def test_batch_group_dedup_equals_per_view_calls(textures):
    views = _make_views(textures, n=7, seed=19)
    o = _ctf.batch_opts(tile_w=8, tile_h=4, mask_dim=11, items_per_fetch=2, ctas_per_sm=4, group_dedup=1)
    fopts = {"tile_w": 8, "tile_h": 4, "mask_dim": 11, "group_dedup": 1}
    st = _ctf.ctf_filter_batch(views, "mask", 5, o, stats=True)
    _ctf.ctf_sync_check()
    singles = []
    for v in views:
        ref, ref_ev, ref_st = _single(v, "mask", 5, fopts)
        singles.append(ref_st)
        H, W = v["height"], v["width"]
        assert np.array_equal(v["out_rgba"].cpu().numpy()[:H, :W].view(np.uint32), ref[:H, :W].view(np.uint32))
        assert np.array_equal(v["out_evals"].cpu().numpy()[:H, :W], ref_ev[:H, :W])
    assert st == _sum_stats(singles)
    assert st["texel_evals_unique"] < st["texel_evals"]


def test_batch_fallback_cplus_equals_per_view_calls(textures):
    views = [v for v in _make_views(textures, n=9, seed=23) if v["kind"] == "block"]
    o = _ctf.batch_opts(tile_w=8, tile_h=4, mask_dim=11, items_per_fetch=2, ctas_per_sm=4, fallback=2)
    fopts = {"tile_w": 8, "tile_h": 4, "mask_dim": 11, "fallback": 2}
    st = _ctf.ctf_filter_batch(views, "mask", 5, o, stats=True)
    _ctf.ctf_sync_check()
    singles = []
    for v in views:
        ref, ref_ev, ref_st = _single(v, "mask", 5, fopts)
        singles.append(ref_st)
        H, W = v["height"], v["width"]
        assert np.array_equal(v["out_rgba"].cpu().numpy()[:H, :W].view(np.uint32), ref[:H, :W].view(np.uint32))
        assert np.array_equal(v["out_evals"].cpu().numpy()[:H, :W], ref_ev[:H, :W])
    assert st == _sum_stats(singles)
    # a learned view refuses the C / C+ fallbacks
    lv = [v for v in _make_views(textures, n=4, seed=23) if v["kind"] != "block"][:1]
    with pytest.raises(_ctf.CtfError):
        _ctf.ctf_filter_batch(lv, "mask", 5, o)


@pytest.mark.parametrize("solo", [1, 400])
def test_batch_solo_views_equal_per_view_calls(textures, solo):
    """Views of at least solo_tiles warp tiles run as their own launches of
    the single-view kernels, the others in the persistent launches: every
    view and the summed counters equal per-view calls either way, directly
    and replayed from a graph (solo 400 puts a learned and two block views
    on their own here)."""
    views = _make_views(textures, n=9, seed=19)
    tiles = [((v["width"] + 7) // 8) * ((v["height"] + 3) // 4) for v in views]
    alone = [t >= solo for t in tiles]
    assert any(alone) and (solo == 1 or not all(alone))
    o = _ctf.batch_opts(tile_w=8, tile_h=4, mask_dim=11, items_per_fetch=2, ctas_per_sm=4, solo_tiles=solo)
    st = _ctf.ctf_filter_batch(views, "mask", 9, o, stats=True)
    _ctf.ctf_sync_check()
    fopts = {"tile_w": 8, "tile_h": 4, "mask_dim": 11}
    singles, refs = [], []
    for v in views:
        ref, ref_ev, ref_st = _single(v, "mask", 9, fopts)
        singles.append(ref_st)
        refs.append((ref, ref_ev))
        H, W = v["height"], v["width"]
        assert np.array_equal(v["out_rgba"].cpu().numpy()[:H, :W].view(np.uint32), ref[:H, :W].view(np.uint32))
        assert np.array_equal(v["out_evals"].cpu().numpy()[:H, :W], ref_ev[:H, :W])
    assert st == _sum_stats(singles)
    for v in views:
        v["out_rgba"].fill_(-1.0)
        v["out_evals"].fill_(7)
    g = _ctf.ctf_batch_graph_create(views, "mask", 9, o)
    try:
        _ctf.ctf_batch_graph_launch(g)
        _ctf.ctf_sync_check()
    finally:
        _ctf.ctf_batch_graph_destroy(g)
    for v, (ref, ref_ev) in zip(views, refs):
        H, W = v["height"], v["width"]
        assert np.array_equal(v["out_rgba"].cpu().numpy()[:H, :W].view(np.uint32), ref[:H, :W].view(np.uint32))
        assert np.array_equal(v["out_evals"].cpu().numpy()[:H, :W], ref_ev[:H, :W])


def test_full_size_uneven_views():
    """The benchmark's batch of 64 uneven views (256..3840 x 256..2160, 179
    Mpixel; 2048^2 block and 4096^2 learned FP16 textures alternating), Mask-11
    with 8x4 tiles: the persistent batch (solo_tiles 0) and the default batch
    (large views in their own launches) both give every view bit for bit as a
    ctf_filter call on it, and 16-row bands of block views equal the oracle run
    on those rows of the view (y_offset)."""
    blocks = synth.random_blocks(2048, 2048, seed=41)
    tb = _ctf.ctf_texture_create(2048, 2048, blocks)
    lat, p = _learned_params(9, 4096, 4096)
    tl = _ctf.ctf_texture_create_mlp(4096, 4096, _ctf.CTF_EVAL_MLP_FP16, lat, *p)
    try:
        raw = synth.uneven_views(64, textures=((2048, 2048), (4096, 4096)))
        views = []
        for i, (sc, ti) in enumerate(raw):
            views.append({"tex": tb if ti == 0 else tl, "sc": sc, "width": sc.W, "height": sc.H, "view_id": i,
                          "uv": torch.from_numpy(sc.uv).cuda(), "jac": torch.from_numpy(sc.jac).cuda(),
                          "coverage": torch.from_numpy(sc.coverage).cuda(),
                          "out_rgba": torch.empty((sc.H, sc.W, 4), device="cuda"),
                          "out_evals": torch.empty((sc.H, sc.W), dtype=torch.uint8, device="cuda")})
        assert sum(v["width"] * v["height"] for v in views) > 150e6
        fo = {"tile_w": 8, "tile_h": 4, "mask_dim": 11}
        ref = []
        for v in views:
            o = torch.empty_like(v["out_rgba"])
            e = torch.empty_like(v["out_evals"])
            _ctf.ctf_filter(v["tex"], v["uv"], v["jac"], v["coverage"], v["width"], v["height"], v["view_id"], "mask",
                            0, fo, o, e)
            ref.append((o, e))
        _ctf.ctf_sync_check()
        for solo in (0, 16384):
            for v in views:
                v["out_rgba"].fill_(-1.0)
                v["out_evals"].fill_(7)
            _ctf.ctf_filter_batch(views, "mask", 0, _ctf.batch_opts(mask_dim=11, solo_tiles=solo))
            _ctf.ctf_sync_check()
            for v, (o, e) in zip(views, ref):
                assert torch.equal(v["out_rgba"].view(torch.int32), o.view(torch.int32)), (solo, v["view_id"])
                assert torch.equal(v["out_evals"], e), (solo, v["view_id"])
        # oracle bands of three block views
        checked = 0
        for v, (o, e) in zip(views, ref):
            if v["tex"] is not tb or v["height"] < 64:
                continue
            sc = v["sc"]
            y0 = (v["height"] // 2) & ~3
            band = slice(y0, y0 + 16)
            r_out, r_ev, _ = oracle.filter_frame(blocks, 2048, 2048, sc.uv[band], sc.jac[band], sc.coverage[band],
                                                 view=v["view_id"], alg=oracle.ALG_MASK, seed=0, mask_dim=11,
                                                 y_offset=y0)
            np.testing.assert_array_equal(e[band].cpu().numpy(), r_ev)
            assert np.array_equal(o[band].cpu().numpy().view(np.uint32), r_out.view(np.uint32))
            checked += 1
            if checked == 3:
                break
        assert checked == 3
    finally:
        _ctf.ctf_texture_destroy(tl)
        _ctf.ctf_texture_destroy(tb)
