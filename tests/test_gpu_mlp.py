"""GPU parity of the learned texel decode (tcgen05 MLP) against the FP64 oracle.

Tolerance, derived from the arithmetic of the FP16 path: the features are
rounded to FP16 and so are both hidden activations (unit roundoff u = 2^-11);
products are exact and sums are FP32 on the tensor cores.  To first order the
output error of a texel is bounded by
    e_f  = u |f|,  e_h1 = u |h1| + |W1| e_f,  e_h2 = u |h2| + |W2| e_h1,
    e_y  = |W3| e_h2
(ReLU and the final clamp are 1-Lipschitz).  Each test allows 1.5 e_y + 1e-5,
computed per texel from the oracle's FP64 activations with the stored
weights.  Texel-evaluation counts must match the oracle bit-exactly: the
selection uses the same FP32 coordinate arithmetic as the exact path.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2506_17770_gb300 import _ctf, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

U16 = 2.0 ** -11
ALGS = {"4tap": 0, "stf": 1, "list_merge": 2, "box": 3, "mask": 4}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_17770_gb300 import build
    build.build()
    oracle.build()


def random_params(seed, Wt, Ht, r0=4, r1=8):
    g = np.random.default_rng(seed)
    lat = [g.normal(0, 1.0, (Ht // r0, Wt // r0, 8)).astype(np.float32),
           g.normal(0, 1.0, (Ht // r1, Wt // r1, 8)).astype(np.float32)]
    w1 = g.normal(0, math.sqrt(2 / 16), (64, 16)).astype(np.float32)
    b1 = g.normal(0, 0.1, 64).astype(np.float32)
    w2 = g.normal(0, math.sqrt(2 / 64), (64, 64)).astype(np.float32)
    b2 = g.normal(0, 0.1, 64).astype(np.float32)
    w3 = g.normal(0, 0.04, (4, 64)).astype(np.float32)
    b3 = np.array([0.5, 0.45, 0.55, 0.9], np.float32)
    return lat, (w1, b1, w2, b2, w3, b3)


class LearnedTex:
    def __init__(self, Wt, Ht, seed=1, mode=_ctf.CTF_EVAL_MLP_FP16):
        self.Wt, self.Ht = Wt, Ht
        lat, p = random_params(seed, Wt, Ht)
        self.h = _ctf.ctf_texture_create_mlp(Wt, Ht, mode, lat, *p)
        st = _ctf.ctf_mlp_export(self.h, (lat[0].shape, lat[1].shape))
        self.stored = st
        self.mlp = oracle.MLP((st["lat0"], st["lat1"]), st["w1"], st["b1"], st["w2"], st["b2"], st["w3"], st["b3"])
        self.bound = self._texel_bounds()

    def _texel_bounds(self):
        st = self.stored
        ys, xs = np.meshgrid(np.arange(self.Ht), np.arange(self.Wt), indexing="ij")
        xs, ys = xs.ravel(), ys.ravel()
        F = np.stack([oracle.mlp_features(self.mlp, self.Wt, self.Ht, int(x), int(y)) for x, y in zip(xs, ys)])
        w1, w2, w3 = (st[k].astype(np.float64) for k in ("w1", "w2", "w3"))
        h1 = np.maximum(F @ w1.T + st["b1"], 0)
        h2 = np.maximum(h1 @ w2.T + st["b2"], 0)
        e_f = U16 * np.abs(F)
        e_h1 = U16 * h1 + e_f @ np.abs(w1).T
        e_h2 = U16 * h2 + e_h1 @ np.abs(w2).T
        e_y = e_h2 @ np.abs(w3).T
        return (1.5 * e_y + 1e-5).reshape(self.Ht, self.Wt, 4)

    def close(self):
        _ctf.ctf_texture_destroy(self.h)


def fp8_weights(st):
    """W_eff = s_o q[o][k] / a_k of an exported E4M3 texture, in FP64."""
    return [(st[f"ws{l}"][:, None] * st[w] / st[f"as{l}"][None, :]).astype(np.float64)
            for l, w in enumerate(("w1", "w2", "w3"))]


def fp8_texel_bound(F, weff, st):
    """Per-texel bound of the E4M3 path for features F (rows): relative
    rounding 2^-4 plus half the subnormal spacing (2^-10 in scaled units) per
    layer input, propagated through |W_eff|, times 2, plus 1e-5."""
    h1 = np.maximum(F @ weff[0].T + st["b1"], 0)
    h2 = np.maximum(h1 @ weff[1].T + st["b2"], 0)
    u = 2.0 ** -4
    e_f = u * np.abs(F) + 2.0 ** -10 * st["as0"]
    e_h1 = u * h1 + 2.0 ** -10 * st["as1"] + e_f @ np.abs(weff[0]).T
    e_h2 = u * h2 + 2.0 ** -10 * st["as2"] + e_h1 @ np.abs(weff[1]).T
    return 2.0 * (e_h2 @ np.abs(weff[2]).T) + 1e-5


def fp8_act_absmax(lat, p, Wt, Ht, xs, ys, margin):
    """Per-channel ranges of the FP32 network's layer inputs over texels
    (xs, ys), times `margin`."""
    full = oracle.MLP((lat[0], lat[1]), *p)
    F = np.stack([oracle.mlp_features(full, Wt, Ht, int(x), int(y)) for x, y in zip(xs, ys)])
    h1 = np.maximum(F @ p[0].T.astype(np.float64) + p[1], 0)
    h2 = np.maximum(h1 @ p[2].T.astype(np.float64) + p[3], 0)
    return [(margin * np.abs(a).max(axis=0) + 1e-3).astype(np.float32) for a in (F, h1, h2)]


class LearnedTexFP8:
    """E4M3 texture of the same random parameters.  The activation ranges are
    those of the FP64 network over every texel (times 1.1), so nothing
    saturates.  Per-texel bound as for FP16, with E4M3's relative rounding
    2^-4 plus half its subnormal spacing (2^-10 in scaled units) per layer
    input, through |W_eff| with W_eff = s_o q[o][k] / a_k as stored."""

    def __init__(self, Wt, Ht, seed=1):
        self.Wt, self.Ht = Wt, Ht
        lat, p = random_params(seed, Wt, Ht)
        ys, xs = np.meshgrid(np.arange(Ht), np.arange(Wt), indexing="ij")
        xs, ys = xs.ravel(), ys.ravel()
        amax = fp8_act_absmax(lat, p, Wt, Ht, xs, ys, 1.1)
        self.h = _ctf.ctf_texture_create_mlp(Wt, Ht, _ctf.CTF_EVAL_MLP_FP8, lat, *p, act_absmax=amax)
        st = _ctf.ctf_mlp_export(self.h, (lat[0].shape, lat[1].shape))
        weff = fp8_weights(st)
        self.mlp = oracle.MLP((st["lat0"], st["lat1"]), weff[0], st["b1"], weff[1], st["b2"], weff[2], st["b3"])
        F = np.stack([oracle.mlp_features(self.mlp, Wt, Ht, int(x), int(y)) for x, y in zip(xs, ys)])
        self.bound = fp8_texel_bound(F, weff, st).reshape(Ht, Wt, 4)

    def close(self):
        _ctf.ctf_texture_destroy(self.h)


@pytest.fixture(scope="module")
def tex64():
    t = LearnedTex(64, 64, seed=1)
    yield t
    t.close()


@pytest.fixture(scope="module")
def tex64_fp8():
    t = LearnedTexFP8(64, 64, seed=1)
    yield t
    t.close()


def test_export_round_trips_fp16(tex64):
    lat, (w1, b1, w2, b2, w3, b3) = random_params(1, 64, 64)
    st = tex64.stored
    np.testing.assert_array_equal(st["w2"], w2.astype(np.float16).astype(np.float32))
    np.testing.assert_array_equal(st["lat1"], lat[1].astype(np.float16).astype(np.float32))
    np.testing.assert_array_equal(st["b2"], b2)


def test_mlp_decode_matches_fp64_oracle(tex64):
    g = np.random.default_rng(4)
    n = 3000
    xy = np.stack([g.integers(-5, 70, n), g.integers(-5, 70, n)], -1).astype(np.int32)
    d_xy = torch.from_numpy(xy).cuda()
    out = torch.full((n, 4), -1.0, device="cuda")
    _ctf.ctf_mlp_decode(tex64.h, d_xy, n, out)
    _ctf.ctf_sync_check()
    got = out.cpu().numpy()
    xc, yc = np.clip(xy[:, 0], 0, 63), np.clip(xy[:, 1], 0, 63)
    ref = oracle.mlp_decode(tex64.mlp, 64, 64, xc, yc)
    tol = tex64.bound[yc, xc]
    err = np.abs(got - ref)
    assert np.all(err <= tol), (err.max(), (err / tol).max())
    assert err.max() > 0  # FP16 rounding is visible: the kernel is not an FP64 copy


def test_mlp_decode_is_row_independent(tex64):
    """A texel's value does not depend on which row of the 128-row tile it
    lands in or on the other rows (needed for collaborative == 4-tap)."""
    g = np.random.default_rng(5)
    base = np.stack([g.integers(0, 64, 200), g.integers(0, 64, 200)], -1).astype(np.int32)
    perm = g.permutation(200)
    outs = []
    for arr in (base, base[perm], np.concatenate([base[:7], base])[7:]):
        d = torch.from_numpy(np.ascontiguousarray(arr)).cuda()
        o = torch.empty((len(arr), 4), device="cuda")
        _ctf.ctf_mlp_decode(tex64.h, d, len(arr), o)
        outs.append(o.cpu().numpy())
    _ctf.ctf_sync_check()
    inv = np.argsort(perm)
    assert np.array_equal(outs[0].view(np.uint32), outs[1][inv].view(np.uint32))
    assert np.array_equal(outs[0].view(np.uint32), outs[2].view(np.uint32))


def _scene(W, H, seed):
    g = np.random.default_rng(seed)
    uv = np.zeros((H, W, 2))
    jac = np.zeros((H, W, 4))
    for ty in range(0, H, 4):
        for tx in range(0, W, 8):
            m = math.exp(g.uniform(math.log(0.6), math.log(8.0)))
            r = g.uniform(0, 2 * math.pi)
            c, s = math.cos(r), math.sin(r)
            o = g.uniform(-2, 62, 2)
            ly, lx = np.meshgrid(np.arange(4) + 0.5, np.arange(8) + 0.5, indexing="ij")
            X = (c * lx - s * ly) / m + o[0]
            Y = (s * lx + c * ly) / m + o[1]
            hh, ww = min(4, H - ty), min(8, W - tx)
            sl = (slice(ty, ty + hh), slice(tx, tx + ww))
            uv[sl + (0,)] = (X / 64)[:hh, :ww]
            uv[sl + (1,)] = (Y / 64)[:hh, :ww]
            jac[sl] = np.array([c / m / 64, s / m / 64, -s / m / 64, c / m / 64])
    cov = (g.uniform(size=(H, W)) > 0.1).astype(np.uint8)
    return uv.astype(np.float32), jac.astype(np.float32), cov


def _pixel_bounds(tex, uv):
    xf = uv[..., 0] * np.float32(tex.Wt) - np.float32(0.5)
    yf = uv[..., 1] * np.float32(tex.Ht) - np.float32(0.5)
    ok = np.isfinite(xf) & np.isfinite(yf) & (np.abs(xf) < 2 ** 22) & (np.abs(yf) < 2 ** 22)
    x0 = np.floor(np.where(ok, xf, 0)).astype(np.int64)
    y0 = np.floor(np.where(ok, yf, 0)).astype(np.int64)
    b = np.zeros(uv.shape[:2] + (4,))
    for dy in (0, 1):
        for dx in (0, 1):
            xx = np.clip(x0 + dx, 0, tex.Wt - 1)
            yy = np.clip(y0 + dy, 0, tex.Ht - 1)
            b = np.maximum(b, tex.bound[yy, xx])
    return b


def gpu_filter(tex, uv, jac, cov, alg, opts=None, seed=0):
    H, W = uv.shape[:2]
    d_uv, d_jac = torch.from_numpy(uv).cuda(), torch.from_numpy(jac).cuda()
    d_cov = None if cov is None else torch.from_numpy(cov).cuda()
    out = torch.full((H, W, 4), -3.0, device="cuda")
    ev = torch.full((H, W), 77, dtype=torch.uint8, device="cuda")
    st = _ctf.ctf_filter(tex.h, d_uv, d_jac, d_cov, W, H, 0, alg, seed, opts, out, ev, stats=True)
    _ctf.ctf_sync_check()
    return out.cpu().numpy(), ev.cpu().numpy(), st


@pytest.mark.parametrize("alg", list(ALGS))
@pytest.mark.parametrize("W,H,seed", [(128, 64, 11), (37, 21, 12)])
def test_learned_filter_matches_fp64_oracle(tex64, alg, W, H, seed):
    uv, jac, cov = _scene(W, H, seed)
    for opts in (None, {"tile_w": 4, "tile_h": 8, "mask_dim": 11}, {"tile_w": 16, "tile_h": 2, "mask_dim": 11}):
        o = {"tile_w": 8, "tile_h": 4, "budget": 32, "mask_dim": 16, "edge_remap": 1}
        o.update(opts or {})
        out, ev, st = gpu_filter(tex64, uv, jac, cov, alg, opts)
        ref, ref_ev, ref_st = oracle.filter_frame_learned_f64(tex64.mlp, 64, 64, uv, jac, cov, alg=ALGS[alg],
                                                              seed=0, **o)
        np.testing.assert_array_equal(ev, ref_ev)
        assert st == ref_st
        tol = _pixel_bounds(tex64, uv)
        err = np.abs(out - ref)
        assert np.all(err <= tol), (alg, opts, err.max())


@pytest.mark.parametrize("alg", list(ALGS))
def test_fp8_filter_matches_fp64_oracle_and_every_kernel_agrees(tex64_fp8, alg):
    """The FP8 E4M3 filter on a ragged view: counts bit-exact and pixels
    within the E4M3 bound of the FP64 oracle; the same call with group_dedup
    and the persistent batch kernel (one role per warp) give the same image
    bitwise."""
    W, H = 133, 70
    uv, jac, cov = _scene(W, H, 17)
    out, ev, st = gpu_filter(tex64_fp8, uv, jac, cov, alg, {"mask_dim": 11})
    ref, ref_ev, ref_st = oracle.filter_frame_learned_f64(tex64_fp8.mlp, 64, 64, uv, jac, cov, alg=ALGS[alg],
                                                          seed=0, mask_dim=11)
    np.testing.assert_array_equal(ev, ref_ev)
    assert st == ref_st
    err = np.abs(out - ref)
    tol = _pixel_bounds(tex64_fp8, uv)
    assert np.all(err <= tol), (alg, err.max(), (err / tol).max())
    assert err.max() > 0  # E4M3 rounding shows
    if alg != "4tap":
        out1 = gpu_filter(tex64_fp8, uv, jac, cov, alg, {"mask_dim": 11, "group_dedup": 1})[0]
        assert np.array_equal(out1.view(np.uint32), out.view(np.uint32))
    view = {"tex": tex64_fp8.h, "uv": torch.from_numpy(uv).cuda(), "jac": torch.from_numpy(jac).cuda(),
            "coverage": torch.from_numpy(cov).cuda(), "width": W, "height": H, "view_id": 0,
            "out_rgba": torch.full((H, W, 4), -1.0, device="cuda"),
            "out_evals": torch.full((H, W), 7, dtype=torch.uint8, device="cuda")}
    stb = _ctf.ctf_filter_batch([view], alg, 0, _ctf.batch_opts(mask_dim=11, solo_tiles=0), stats=True)
    _ctf.ctf_sync_check()
    assert np.array_equal(view["out_rgba"].cpu().numpy().view(np.uint32), out.view(np.uint32))
    np.testing.assert_array_equal(view["out_evals"].cpu().numpy(), ev)
    assert stb == st


@pytest.mark.parametrize("W,H", [(1, 1), (1, 37), (37, 1), (8, 4), (9, 5), (64, 3)])
@pytest.mark.parametrize("alg", ["stf", "box", "mask", "list_merge"])
def test_learned_tiny_and_uncovered_views(tex64, W, H, alg):
    """Views of one pixel, one row, one column, one tile and a few ragged
    tiles (a group of 8 tiles with most slots empty): counts and statistics
    bit-exact, pixels within the FP16 bound; with nothing covered, zeros."""
    uv, jac, cov = _scene(W, H, 5)
    cov[:] = 1
    out, ev, st = gpu_filter(tex64, uv, jac, cov, alg, {"mask_dim": 11})
    ref, ref_ev, ref_st = oracle.filter_frame_learned_f64(tex64.mlp, 64, 64, uv, jac, cov, alg=ALGS[alg], seed=0,
                                                          mask_dim=11)
    np.testing.assert_array_equal(ev, ref_ev)
    assert st == ref_st
    assert np.all(np.abs(out - ref) <= _pixel_bounds(tex64, uv))
    out, ev, st = gpu_filter(tex64, uv, jac, np.zeros_like(cov), alg, {"mask_dim": 11})
    assert st["pixels_active"] == 0 and st["tiles_empty"] == st["tiles_total"] > 0
    assert not out.any() and not ev.any()


def test_learned_success_equals_learned_4tap_bitwise(tex64):
    sc = synth.magnified_plane(128, 128, 64, 64, scale=0.25)
    ref = gpu_filter(tex64, sc.uv, sc.jac, None, "4tap")[0]
    for alg in ("box", "mask", "list_merge"):
        out, ev, st = gpu_filter(tex64, sc.uv, sc.jac, None, alg)
        assert st["tiles_success"] == st["tiles_total"]
        assert np.array_equal(out.view(np.uint32), ref.view(np.uint32)), alg
        assert st["texel_evals"] < 0.75 * st["pixels_active"]


@pytest.mark.parametrize("alg", ["stf", "list_merge", "box", "mask"])
@pytest.mark.parametrize("W,H,seed", [(128, 64, 11), (37, 21, 12)])
def test_group_dedup_changes_only_the_evaluation_count(tex64, alg, W, H, seed):
    """group_dedup evaluates each distinct texel of a group of 8 tiles once:
    the image (bitwise) and the per-pixel counts stay those of the per-warp
    method, and texel_evals_unique equals the oracle's grouped count."""
    uv, jac, cov = _scene(W, H, seed)
    out0, ev0, st0 = gpu_filter(tex64, uv, jac, cov, alg, {"mask_dim": 11})
    out1, ev1, st1 = gpu_filter(tex64, uv, jac, cov, alg, {"mask_dim": 11, "group_dedup": 1})
    assert np.array_equal(out1.view(np.uint32), out0.view(np.uint32))
    np.testing.assert_array_equal(ev1, ev0)
    ref_st = oracle.filter_frame_learned_f64(tex64.mlp, 64, 64, uv, jac, cov, alg=ALGS[alg], seed=0, mask_dim=11,
                                             group_tiles=8)[2]
    assert st1 == ref_st
    assert st1["texel_evals_unique"] <= st0["texel_evals_unique"] == st0["texel_evals"]


def test_group_dedup_on_a_magnified_plane(tex64):
    sc = synth.magnified_plane(256, 128, 64, 64, scale=0.25)
    out0, _, st0 = gpu_filter(tex64, sc.uv, sc.jac, None, "box")
    out1, _, st1 = gpu_filter(tex64, sc.uv, sc.jac, None, "box", {"group_dedup": 1})
    assert np.array_equal(out1.view(np.uint32), out0.view(np.uint32))
    ref_st = oracle.filter_frame_learned_f64(tex64.mlp, 64, 64, sc.uv, sc.jac, None, alg=ALGS["box"], seed=0,
                                             group_tiles=8)[2]
    assert st1 == ref_st
    # neighbouring 8x4 tiles share the texels along their common edges
    assert st1["texel_evals_unique"] < 0.8 * st1["texel_evals"]


EXT_OPTS = [{"fallback": 1}, {"fallback": 2}, {"texels_per_lane": 2, "budget": 64},
            {"fallback": 2, "texels_per_lane": 2, "budget": 64, "mask_dim": 11}]


@pytest.mark.parametrize("opts", EXT_OPTS, ids=["C", "C+", "two", "C+two"])
@pytest.mark.parametrize("alg", ["list_merge", "box", "mask"])
@pytest.mark.parametrize("fp8", [False, True])
def test_learned_extensions_match_fp64_oracle(tex64, tex64_fp8, alg, opts, fp8):
    """Fallbacks C and C+ (Sec. 3.4) and two texels per lane (Sec. 5) on a
    learned texture: per-pixel counts and statistics bit-exact against the
    FP64 oracle, pixels within the texel bound of the decode.  Eq. 1 blends a
    pixel's produced footprint texels with weights that sum to one (the
    bilinear weights present plus (1 - S_w) / N each), and the success path
    is the bilinear filter, so a pixel's error is at most the largest error
    of its footprint texels, the bound _pixel_bounds takes.  The view holds
    over-budget and minified tiles and a ragged edge."""
    tex = tex64_fp8 if fp8 else tex64
    W, H = 133, 70
    uv, jac, cov = _scene(W, H, 23)
    o = {"tile_w": 8, "tile_h": 4, "budget": 32, "mask_dim": 16, "edge_remap": 1}
    o.update(opts)
    out, ev, st = gpu_filter(tex, uv, jac, cov, alg, opts, seed=5)
    ref, ref_ev, ref_st = oracle.filter_frame_learned_f64(
        tex.mlp, 64, 64, uv, jac, cov, alg=ALGS[alg], seed=5, tile_w=o["tile_w"], tile_h=o["tile_h"],
        budget=o["budget"], mask_dim=o["mask_dim"], edge_remap=o["edge_remap"], fallback=o.get("fallback", 0),
        texels_per_lane=o.get("texels_per_lane", 1))
    np.testing.assert_array_equal(ev, ref_ev)
    assert st == ref_st
    if "fallback" in opts and "texels_per_lane" not in opts:
        assert st["tiles_fallback_budget"] > 0
    assert st["tiles_fallback_minified"] > 0
    err = np.abs(out - ref)
    tol = _pixel_bounds(tex, uv)
    assert np.all(err <= tol), (alg, opts, err.max(), (err / tol).max())


def test_learned_two_texels_per_lane_equal_learned_4tap_on_success(tex64):
    """Where a tile succeeds with two texels per lane, its pixels equal the
    learned per-pixel 4-tap image bit for bit: the same texel values (rows
    of the same chain) and the same filter arithmetic."""
    W, H = 133, 70
    uv, jac, cov = _scene(W, H, 29)
    two, ev, st = gpu_filter(tex64, uv, jac, cov, "mask", {"texels_per_lane": 2, "budget": 64})
    four = gpu_filter(tex64, uv, jac, cov, "4tap")[0]
    _, _, _, tp, _ = oracle.filter_frame(synth.random_blocks(64, 64), 64, 64, uv, jac, cov, alg=4,
                                         texels_per_lane=2, budget=64, want_tiles=True)
    tiles_x = (W + 7) // 8
    checked = 0
    for t, path in enumerate(tp):
        if path != oracle.PATH_SUCCESS:
            continue
        by, bx = divmod(t, tiles_x)
        sl = (slice(4 * by, 4 * by + 4), slice(8 * bx, 8 * bx + 8))
        assert np.array_equal(two[sl].view(np.uint32), four[sl].view(np.uint32)), t
        checked += 1
    assert checked > 100 and st["tiles_success"] == checked


@pytest.mark.parametrize("md", [16, 11])
def test_learned_two_texels_per_lane_on_rotated_quads(tex64, md):
    """Two texels per lane on head-on quads rotated by 0..90 degrees just
    above magnification 1 (Sec. 5): Mask tiles of up to 54 texels whose
    bounding boxes span more than 64 positions, so the texel ranks 32..63
    (the second round) are in use.  Counts and statistics equal the FP64
    oracle's, the pixels lie within the decode bound, and every tile
    succeeds."""
    q = synth.rotated_quad_tiles(1.001, np.arange(0, 91, 3.0), 8, Wt=64, Ht=64)
    # the quads sit near texel 1024; move them to the middle of the 64^2 texture
    uv = (q.uv.astype(np.float64) - 996.0 / 64.0).astype(np.float32)
    jac = q.jac.astype(np.float32)
    opts = {"texels_per_lane": 2, "budget": 64, "mask_dim": md}
    out, ev, st = gpu_filter(tex64, uv, jac, None, "mask", opts)
    ref, ref_ev, ref_st = oracle.filter_frame_learned_f64(tex64.mlp, 64, 64, uv, jac, None, alg=ALGS["mask"], seed=0,
                                                          budget=64, mask_dim=md, texels_per_lane=2)
    np.testing.assert_array_equal(ev, ref_ev)
    assert st == ref_st
    assert st["tiles_success"] == st["tiles_total"]
    per_tile = ev.reshape(-1, 4, 8).sum(axis=(1, 2))
    assert per_tile.max() > 32 and np.count_nonzero(per_tile > 32) >= 20
    err = np.abs(out - ref)
    assert np.all(err <= _pixel_bounds(tex64, uv)), err.max()


def test_learned_extensions_refuse_group_dedup(tex64):
    uv, jac, cov = _scene(37, 21, 12)
    with pytest.raises(_ctf.CtfError) as ei:
        gpu_filter(tex64, uv, jac, cov, "mask", {"fallback": 1, "group_dedup": 1})
    assert ei.value.status == _ctf.CTF_ERR_UNSUPPORTED


@pytest.mark.parametrize("dedup", [0, 1])
@pytest.mark.parametrize("alg", ["stf", "box", "mask"])
def test_specialised_warps_equal_the_batch_kernel(tex64, alg, dedup):
    """The single-view learned filter runs step 1 and the gather in producer
    warps and the MMA chains in a consumer warpgroup, handing groups over
    through two stages of buffers; the persistent batch kernel does all of it
    in every warp.  On a ragged view of several groups per CTA, with a band
    of uncovered pixels (groups with no texel to evaluate) and the coverage
    array at an odd byte offset, both give the same image and counts, with
    and without group_dedup."""
    W, H = 1283, 797
    uv, jac, cov = _scene(W, H, 21)
    cov[:, :300] = 0
    big = torch.zeros(W * H + 8, dtype=torch.uint8, device="cuda")
    big[3:3 + W * H] = torch.from_numpy(cov.reshape(-1)).cuda()
    d_cov = big[3:3 + W * H].view(H, W)
    d_uv, d_jac = torch.from_numpy(uv).cuda(), torch.from_numpy(jac).cuda()
    out = torch.full((H, W, 4), -3.0, device="cuda")
    ev = torch.full((H, W), 77, dtype=torch.uint8, device="cuda")
    st = _ctf.ctf_filter(tex64.h, d_uv, d_jac, d_cov, W, H, 5, alg, 9, {"mask_dim": 11, "group_dedup": dedup}, out, ev,
                         stats=True)
    view = {"tex": tex64.h, "uv": d_uv, "jac": d_jac, "coverage": d_cov, "width": W, "height": H, "view_id": 5,
            "out_rgba": torch.full((H, W, 4), -1.0, device="cuda"),
            "out_evals": torch.full((H, W), 7, dtype=torch.uint8, device="cuda")}
    o = _ctf.batch_opts(mask_dim=11, solo_tiles=0, group_dedup=dedup)
    stb = _ctf.ctf_filter_batch([view], alg, 9, o, stats=True)
    _ctf.ctf_sync_check()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), view["out_rgba"].cpu().numpy().view(np.uint32))
    np.testing.assert_array_equal(ev.cpu().numpy(), view["out_evals"].cpu().numpy())
    assert st == stb
    assert st["pixels_active"] == int(cov.sum())
    assert st["tiles_empty"] >= 300 // 8 * (H // 4)


@pytest.mark.parametrize("fp8", [False, True])
def test_learned_full_view_bands_match_fp64_oracle(fp8):
    """The 3840x2160 learned view of the benchmark (4096^2 texture, latent
    grids 1024^2 and 512^2, magnification 1 to 16) filtered with Mask-11 in
    the launch the bench times (one launch over the whole view, 8x4 tiles),
    FP16 and FP8.  Three bands of 16 rows (top, middle, bottom) against the
    FP64 oracle run on those rows alone (y_offset keeps the STF draws of the
    whole view): counts bit-exact, pixels within the FP16 (or E4M3) bound of
    their footprint's texels.  The FP8 activation ranges come from 20,000
    sampled texels, times 3, so that no activation saturates."""
    Wt = Ht = 4096
    lat, p = random_params(7, Wt, Ht)
    if fp8:
        g = np.random.default_rng(11)
        amax = fp8_act_absmax(lat, p, Wt, Ht, g.integers(0, Wt, 20000), g.integers(0, Ht, 20000), 3.0)
        h = _ctf.ctf_texture_create_mlp(Wt, Ht, _ctf.CTF_EVAL_MLP_FP8, lat, *p, act_absmax=amax)
    else:
        h = _ctf.ctf_texture_create_mlp(Wt, Ht, _ctf.CTF_EVAL_MLP_FP16, lat, *p)
    try:
        st = _ctf.ctf_mlp_export(h, (lat[0].shape, lat[1].shape))
        weff = fp8_weights(st) if fp8 else [st[k].astype(np.float64) for k in ("w1", "w2", "w3")]
        mlp = oracle.MLP((st["lat0"], st["lat1"]), weff[0], st["b1"], weff[1], st["b2"], weff[2], st["b3"])
        sc = synth.perspective_view(3840, 2160, Wt, Ht, 1.0, 16.0, seed=2)
        W, H = sc.W, sc.H
        d_uv, d_jac, d_cov = (torch.from_numpy(a).cuda() for a in (sc.uv, sc.jac, sc.coverage))
        out = torch.full((H, W, 4), -3.0, device="cuda")
        ev = torch.full((H, W), 77, dtype=torch.uint8, device="cuda")
        _ctf.ctf_filter(h, d_uv, d_jac, d_cov, W, H, 0, "mask", 0, {"mask_dim": 11}, out, ev)
        _ctf.ctf_sync_check()
        out, ev = out.cpu().numpy(), ev.cpu().numpy()
        w1, w2, w3 = weff
        for y0 in (0, 1000, H - 16):
            band = slice(y0, y0 + 16)
            ref, ref_ev, _ = oracle.filter_frame_learned_f64(mlp, Wt, Ht, sc.uv[band], sc.jac[band],
                                                             sc.coverage[band], alg=ALGS["mask"], mask_dim=11,
                                                             y_offset=y0)
            np.testing.assert_array_equal(ev[band], ref_ev)
            # bound of every texel of the band's 2x2 footprints
            uv = sc.uv[band]
            x0 = np.floor(uv[..., 0] * np.float32(Wt) - np.float32(0.5)).astype(np.int64)
            y0_ = np.floor(uv[..., 1] * np.float32(Ht) - np.float32(0.5)).astype(np.int64)
            taps = [(np.clip(x0 + dx, 0, Wt - 1), np.clip(y0_ + dy, 0, Ht - 1)) for dy in (0, 1) for dx in (0, 1)]
            keys = np.unique(np.concatenate([ty.ravel() * Wt + tx.ravel() for tx, ty in taps]))
            F = np.stack([oracle.mlp_features(mlp, Wt, Ht, int(k % Wt), int(k // Wt)) for k in keys])
            if fp8:
                kb = fp8_texel_bound(F, weff, st)
            else:
                h1 = np.maximum(F @ w1.T + st["b1"], 0)
                h2 = np.maximum(h1 @ w2.T + st["b2"], 0)
                e_h1 = U16 * h1 + (U16 * np.abs(F)) @ np.abs(w1).T
                e_h2 = U16 * h2 + e_h1 @ np.abs(w2).T
                kb = 1.5 * (e_h2 @ np.abs(w3).T) + 1e-5
            tol = np.zeros(uv.shape[:2] + (4,))
            for tx, ty in taps:
                tol = np.maximum(tol, kb[np.searchsorted(keys, ty * Wt + tx)])
            err = np.abs(out[band].astype(np.float64) - ref)
            assert (sc.coverage[band] != 0).sum() > 0.8 * 16 * W
            assert np.all(err <= tol), (y0, err.max(), (err / tol).max())
    finally:
        _ctf.ctf_texture_destroy(h)


@pytest.mark.parametrize("alg", ["stf", "mask"])
def test_learned_host_entry_point_matches_device(tex64, alg):
    """ctf_filter_host on a learned texture, in row bands (more than 2^20
    pixels): image and counts equal one ctf_filter call on the whole view."""
    W, H = 1400, 800
    uv, jac, cov = _scene(W, H, 31)
    out_d, ev_d, st_d = gpu_filter(tex64, uv, jac, cov, alg, {"mask_dim": 11}, seed=5)
    assert st_d["tiles_fallback_minified"] + st_d["tiles_direct"] > 0
    h = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (uv, jac, cov)]
    out = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
    ev = torch.empty((H, W), dtype=torch.uint8).pin_memory()
    st = _ctf.ctf_filter_host(tex64.h, h[0], h[1], h[2], W, H, 0, alg, 5, {"mask_dim": 11}, out, ev, stats=True)
    assert st == st_d
    assert np.array_equal(out.numpy().view(np.uint32), out_d.view(np.uint32))
    assert np.array_equal(ev.numpy(), ev_d)


def test_bounded_wait_gives_up_and_the_context_stays_usable(tex64):
    """A kernel whose mbarrier wait nobody completes gives up after its bound,
    records CTF_ERR_TIMEOUT for the next ctf_sync_check (which clears it), and
    the next filter call runs and gives its usual result."""
    uv, jac, cov = _scene(37, 21, 12)
    before = gpu_filter(tex64, uv, jac, cov, "mask", {"mask_dim": 11})
    _ctf.ctf_selftest_bounded_wait(1 << 12)
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_sync_check()
    assert ei.value.status == _ctf.CTF_ERR_TIMEOUT
    _ctf.ctf_sync_check()  # the record is cleared
    after = gpu_filter(tex64, uv, jac, cov, "mask", {"mask_dim": 11})
    assert np.array_equal(after[0].view(np.uint32), before[0].view(np.uint32))
    assert np.array_equal(after[1], before[1]) and after[2] == before[2]
