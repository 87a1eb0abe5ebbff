"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-type the oracle's formulas: each compares it with a published
value, an independent library routine (numpy's Philox, scipy's bilinear
interpolation, numpy matmul), a closed form, an invariant or brute force.
"""
import math
import os

import numpy as np
import pytest

from paper_2506_17770_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]


# ---------------------------------------------------------------------------
# Philox
# ---------------------------------------------------------------------------
def test_philox4x32_known_answers(oracle_lib):
    rows = _read_lines("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle_lib.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)), ((5, 7, 11, 13), (123456789, 987654321)),
                                     ((2**64 - 2, 1, 2, 3), (2**63 + 5, 77))])
def test_philox_round_structure_matches_numpy(oracle_lib, ctr, key):
    """numpy's Philox bit generator is Philox4x64-10; it increments the counter
    before each block.  Agreement pins the round function and key schedule that
    the oracle's 4x32 variant shares (only word size and constants differ)."""
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    got = bg.random_raw(4)
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64
    if c[0] == 0:
        c[1] += 1
    ours = oracle_lib.philox4x64_10(c, key)
    assert [int(x) for x in ours] == [int(x) for x in got]


# ---------------------------------------------------------------------------
# Bijection h (Sec. 3.3, Fig. 3)
# ---------------------------------------------------------------------------
def test_bijection_fig3(oracle_lib):
    rows = [r for r in _read_lines("paper_values.txt") if r[0] == "fig3"]
    assert len(rows) == 6
    for _, mask, fn, arg, want in rows:
        B = int(mask, 2)
        got = oracle_lib.h(int(arg), B) if fn == "h" else oracle_lib.hinv(int(arg), B)
        assert got == int(want), (mask, fn, arg)


def test_bijection_inverse_on_random_masks(oracle_lib):
    g = np.random.default_rng(5)
    for _ in range(200):
        B = int(g.integers(0, 2**63)) | (int(g.integers(0, 2**63)) << 63) | (int(g.integers(0, 2**63)) << 126)
        n = bin(B).count("1")
        positions = [oracle_lib.h(i, B) for i in range(n)]
        # brute force: positions of the set bits in increasing order
        assert positions == [t for t in range(256) if (B >> t) & 1]
        for i, t in enumerate(positions):
            assert oracle_lib.hinv(t, B) == i
        assert oracle_lib.h(n, B) == -1


# ---------------------------------------------------------------------------
# Block decode: hand-computed examples
# ---------------------------------------------------------------------------
def test_block_decode_hand_examples(oracle_lib):
    rows = _read_lines("block_decode_examples.txt")
    tex = None
    n_checked = 0
    for r in rows:
        if r[0] == "texture":
            tex = [int(r[1]), int(r[2]), []]
        elif r[0] == "block":
            rec = np.zeros(1, dtype=[("c0", "<u2"), ("c1", "<u2"), ("ix", "<u4")])
            rec["c0"], rec["c1"], rec["ix"] = int(r[1], 16), int(r[2], 16), int(r[3], 16)
            tex[2].append(rec.view(np.uint8))
        elif r[0] == "q":
            blocks = np.concatenate(tex[2])
            x, y = int(r[1]), int(r[2])
            got = oracle_lib.decode_rgba8(blocks, tex[0], tex[1], x, y)
            assert list(got) == [int(v) for v in r[3:7]], (r, list(got))
            n_checked += 1
    assert n_checked == 13


# ---------------------------------------------------------------------------
# Per-pixel bilinear against scipy (independent library routine)
# ---------------------------------------------------------------------------
def _decoded_image(oracle_lib, blocks, Wt, Ht):
    img = np.zeros((Ht, Wt, 4), np.float64)
    for y in range(Ht):
        for x in range(Wt):
            img[y, x] = oracle_lib.decode_rgba8(blocks, Wt, Ht, x, y)
    return img / 255.0


@pytest.mark.parametrize("Wt,Ht", [(16, 16), (32, 8), (8, 24)])
def test_4tap_matches_scipy_bilinear(oracle_lib, Wt, Ht):
    from scipy.ndimage import map_coordinates
    blocks = synth.random_blocks(Wt, Ht, seed=11)
    img = _decoded_image(oracle_lib, blocks, Wt, Ht)
    g = np.random.default_rng(3)
    W, H = 24, 12
    # UVs partly outside [0,1] so clamp-to-edge is exercised
    uv = g.uniform(-0.2, 1.2, (H, W, 2)).astype(np.float32)
    jac = np.zeros((H, W, 4), np.float32)
    out, ev, st = oracle_lib.filter_frame(blocks, Wt, Ht, uv, jac, alg=oracle_lib.ALG_4TAP)
    assert st["pixels_active"] == W * H and np.all(ev == 4)
    # the same FP32 texel-space coordinates (uv * dim - 0.5, IEEE float32 ops)
    xf = (uv[..., 0] * np.float32(Wt)) - np.float32(0.5)
    yf = (uv[..., 1] * np.float32(Ht)) - np.float32(0.5)
    for ch in range(4):
        ref = map_coordinates(img[..., ch], [yf.astype(np.float64).ravel(), xf.astype(np.float64).ravel()],
                              order=1, mode="nearest").reshape(H, W)
        np.testing.assert_allclose(out[..., ch], ref, rtol=0, atol=2e-6)


def test_bspline_matches_scipy(oracle_lib):
    """Per-pixel bicubic with the cubic B-spline (Sec. 4.2) is scipy's order-3
    B-spline applied to the texel samples without prefiltering, clamped to
    the edge, at the same FP32 texel coordinates."""
    from scipy.ndimage import map_coordinates
    o = oracle_lib
    Wt, Ht = 32, 16
    blocks = synth.random_blocks(Wt, Ht, seed=12)
    img = _decoded_image(o, blocks, Wt, Ht)
    g = np.random.default_rng(4)
    W, H = 24, 12
    uv = g.uniform(-0.2, 1.2, (H, W, 2)).astype(np.float32)
    jac = np.zeros((H, W, 4), np.float32)
    out, ev, st = o.filter_frame(blocks, Wt, Ht, uv, jac, alg=o.ALG_4TAP, filter=o.FILTER_BSPLINE)
    assert np.all(ev == 16)
    xf = (uv[..., 0] * np.float32(Wt)) - np.float32(0.5)
    yf = (uv[..., 1] * np.float32(Ht)) - np.float32(0.5)
    for ch in range(4):
        ref = map_coordinates(img[..., ch], [yf.astype(np.float64).ravel(), xf.astype(np.float64).ravel()],
                              order=3, mode="nearest", prefilter=False).reshape(H, W)
        np.testing.assert_allclose(out[..., ch], ref, rtol=0, atol=4e-6)


def test_catmull_rom_closed_forms(oracle_lib):
    """Catmull-Rom interpolates: at texel centres (s = t = 0) the output is
    the texel itself, bitwise; halfway between centres its weights per axis
    are (-1, 9, 9, -1) / 16, so the output is that dyadic blend of the 4x4
    texels (exact rational arithmetic here)."""
    from fractions import Fraction
    o = oracle_lib
    Wt = Ht = 16
    blocks = synth.random_blocks(Wt, Ht, seed=21)
    img = _decoded_image(o, blocks, Wt, Ht)
    xs, ys = np.meshgrid(np.arange(3, 12), np.arange(3, 12))
    uv = np.stack([(xs + 0.5) / Wt, (ys + 0.5) / Ht], axis=-1).astype(np.float32)
    jac = np.zeros(uv.shape[:2] + (4,), np.float32)
    out = o.filter_frame(blocks, Wt, Ht, uv, jac, alg=o.ALG_4TAP, filter=o.FILTER_CATMULL_ROM)[0]
    assert np.array_equal(out.view(np.uint32), img[ys, xs].astype(np.float32).view(np.uint32))
    uv = np.stack([(xs + 1.0) / Wt, (ys + 1.0) / Ht], axis=-1).astype(np.float32)
    out = o.filter_frame(blocks, Wt, Ht, uv, jac, alg=o.ALG_4TAP, filter=o.FILTER_CATMULL_ROM)[0]
    wv = [Fraction(-1, 16), Fraction(9, 16), Fraction(9, 16), Fraction(-1, 16)]
    dec = [[[Fraction(int(v), 255) for v in o.decode_rgba8(blocks, Wt, Ht, x, y)] for x in range(Wt)]
           for y in range(Ht)]
    for (y, x) in [(3, 3), (5, 8), (10, 11), (7, 4)]:
        for ch in range(4):
            exact = sum(wv[i] * wv[j] * dec[y - 1 + j][x - 1 + i][ch] for i in range(4) for j in range(4))
            assert abs(float(exact) - float(out[y - 3, x - 3, ch])) <= 3e-7, (y, x, ch)


def test_4tap_closed_form_at_texel_centres_and_midpoints(oracle_lib):
    """s,t = 0 returns the texel itself; s,t = 1/2 returns the mean of the 2x2."""
    Wt = Ht = 16
    blocks = synth.random_blocks(Wt, Ht, seed=12)
    img = _decoded_image(oracle_lib, blocks, Wt, Ht)
    xs, ys = np.meshgrid(np.arange(2, 12), np.arange(3, 9))
    uv_c = np.stack([(xs + 0.5) / Wt, (ys + 0.5) / Ht], -1).astype(np.float32)
    uv_m = np.stack([(xs + 1.0) / Wt, (ys + 1.0) / Ht], -1).astype(np.float32)
    jac = np.zeros(uv_c.shape[:2] + (4,), np.float32)
    out_c, _, _ = oracle_lib.filter_frame(blocks, Wt, Ht, uv_c, jac, alg=oracle_lib.ALG_4TAP)
    out_m, _, _ = oracle_lib.filter_frame(blocks, Wt, Ht, uv_m, jac, alg=oracle_lib.ALG_4TAP)
    np.testing.assert_array_equal(out_c, img[ys, xs].astype(np.float32))
    mean = (img[ys, xs] + img[ys, xs + 1] + img[ys + 1, xs] + img[ys + 1, xs + 1]) / 4
    np.testing.assert_allclose(out_m, mean, atol=1e-7)


# ---------------------------------------------------------------------------
# Collaborative algorithms: invariants
# ---------------------------------------------------------------------------
def _scene_mix(seed=4, W=96, H=64):
    """Random per-tile rotations and magnifications, some coverage holes."""
    g = np.random.default_rng(seed)
    uv = np.zeros((H, W, 2))
    jac = np.zeros((H, W, 4))
    for ty in range(H // 4):
        for tx in range(W // 8):
            m = math.exp(g.uniform(math.log(0.7), math.log(6.0)))
            r = g.uniform(0, 2 * math.pi)
            c, s = math.cos(r), math.sin(r)
            o = g.uniform(20, 40, 2)
            ly, lx = np.meshgrid(np.arange(4) + 0.5, np.arange(8) + 0.5, indexing="ij")
            X = (c * lx - s * ly) / m + o[0]
            Y = (s * lx + c * ly) / m + o[1]
            sl = (slice(ty * 4, ty * 4 + 4), slice(tx * 8, tx * 8 + 8))
            uv[sl + (0,)] = X / 64
            uv[sl + (1,)] = Y / 64
            jac[sl] = np.array([c / m / 64, s / m / 64, -s / m / 64, c / m / 64])
    cov = (g.uniform(size=(H, W)) > 0.15).astype(np.uint8)
    return uv.astype(np.float32), jac.astype(np.float32), cov


@pytest.mark.parametrize("alg", ["box", "mask16", "mask11", "list"])
def test_success_path_reproduces_bilinear_bitwise(oracle_lib, alg):
    o = oracle_lib
    blocks = synth.random_blocks(64, 64, seed=13)
    uv, jac, cov = _scene_mix()
    a = {"box": o.ALG_BOX, "mask16": o.ALG_MASK, "mask11": o.ALG_MASK, "list": o.ALG_LIST_MERGE}[alg]
    md = 11 if alg == "mask11" else 16
    ref, ev_ref, _ = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=o.ALG_4TAP)
    out, ev, st, tp, tn = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=a, mask_dim=md, want_tiles=True)
    assert st["tiles_success"] > 20 and st["tiles_fallback_budget"] > 5
    H, W = uv.shape[:2]
    tiles_x = W // 8
    for tid in np.nonzero(tp == o.PATH_SUCCESS)[0]:
        ty, tx = divmod(int(tid), tiles_x)
        sl = (slice(ty * 4, ty * 4 + 4), slice(tx * 8, tx * 8 + 8))
        np.testing.assert_array_equal(out[sl], ref[sl])
        # texel i is produced by the i-th active lane: the first n active lanes count 1
        act = cov[sl].ravel() != 0
        cnt = ev[sl].ravel()
        n = int(tn[tid])
        producers = np.nonzero(act)[0][:n]
        expect = np.zeros(32, np.uint8)
        expect[producers] = 1
        np.testing.assert_array_equal(cnt, expect)
    # fallback tiles: every active lane evaluates exactly one texel
    for tid in np.nonzero(tp == o.PATH_FALLBACK_BUDGET)[0]:
        ty, tx = divmod(int(tid), tiles_x)
        sl = (slice(ty * 4, ty * 4 + 4), slice(tx * 8, tx * 8 + 8))
        np.testing.assert_array_equal(ev[sl], (cov[sl] != 0).astype(np.uint8))
    assert st["texel_evals"] == int(ev.sum())


def test_set_sizes_and_nested_success(oracle_lib):
    """Box n = bbox area >= exact unique count (List Merge) = Mask popcount
    whenever the bbox fits the mask; successes nest Box <= Mask <= List."""
    o = oracle_lib
    blocks = synth.random_blocks(64, 64, seed=13)
    uv, jac, cov = _scene_mix(seed=9)
    res = {}
    for name, a, md in (("box", o.ALG_BOX, 16), ("mask", o.ALG_MASK, 16), ("list", o.ALG_LIST_MERGE, 16)):
        _, _, _, tp, tn = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=a, mask_dim=md, want_tiles=True)
        res[name] = (tp, tn)
    tpb, tnb = res["box"]
    tpm, tnm = res["mask"]
    tpl, tnl = res["list"]
    fit = tnm >= 0
    assert fit.sum() > 50
    np.testing.assert_array_equal(tnm[fit], tnl[fit])
    assert np.all(tnb[tnl > 0] >= tnl[tnl > 0])
    sb, sm, sl = (tpb == o.PATH_SUCCESS), (tpm == o.PATH_SUCCESS), (tpl == o.PATH_SUCCESS)
    assert np.all(~sb | sm) and np.all(~sm | sl)
    assert sl.sum() > sm.sum() >= sb.sum() > 0 or sl.sum() >= sm.sum() > sb.sum() > 0


def test_group_distinct_texels_brute_force(oracle_lib):
    """Groups of 8 consecutive tiles evaluating each distinct clamped texel
    once (the shared-memory extension of Sec. 6): on a magnified plane every
    Box tile succeeds and evaluates its whole bounding box, so the grouped
    count is the size of the union of the clamped boxes, which numpy computes
    here from the FP32 texel coordinates.  The plane starts 3 texels left of
    the texture, so clamping merges texels too."""
    o = oracle_lib
    Wt = Ht = 64
    blocks = synth.random_blocks(Wt, Ht, seed=17)
    sc = synth.magnified_plane(96, 40, Wt, Ht, scale=0.25, seed=5)
    uv = sc.uv.copy()
    uv[..., 0] -= np.float32(3.0 / Wt)
    cov = np.ones((40, 96), np.uint8)
    _, ev, st, tp, _ = o.filter_frame(blocks, Wt, Ht, uv, sc.jac, cov, alg=o.ALG_BOX, group_tiles=8,
                                      want_tiles=True)
    assert np.all(tp == o.PATH_SUCCESS)
    xf = uv[..., 0] * np.float32(Wt) - np.float32(0.5)
    yf = uv[..., 1] * np.float32(Ht) - np.float32(0.5)
    ulx, uly = np.floor(xf).astype(int), np.floor(yf).astype(int)
    tiles_x, tiles_y = 96 // 8, 40 // 4
    groups = {}
    for ty in range(tiles_y):
        for tx in range(tiles_x):
            sl = (slice(ty * 4, ty * 4 + 4), slice(tx * 8, tx * 8 + 8))
            x0, x1 = ulx[sl].min(), ulx[sl].max() + 1
            y0, y1 = uly[sl].min(), uly[sl].max() + 1
            texels = {(min(max(x, 0), Wt - 1), min(max(y, 0), Ht - 1))
                      for x in range(x0, x1 + 1) for y in range(y0, y1 + 1)}
            groups.setdefault((ty * tiles_x + tx) // 8, set()).update(texels)
    assert st["texel_evals_unique"] == sum(len(g) for g in groups.values())
    assert st["texel_evals_unique"] < st["texel_evals"] == int(ev.sum())
    # one tile per group: only the clamping merges texels; no grouping: the per-warp count
    st1 = o.filter_frame(blocks, Wt, Ht, uv, sc.jac, cov, alg=o.ALG_BOX, group_tiles=1)[2]
    st0 = o.filter_frame(blocks, Wt, Ht, uv, sc.jac, cov, alg=o.ALG_BOX)[2]
    assert st["texel_evals_unique"] < st1["texel_evals_unique"] < st0["texel_evals_unique"] == st0["texel_evals"]
    # Mask produces a subset of each box: never more distinct texels
    stm = o.filter_frame(blocks, Wt, Ht, uv, sc.jac, cov, alg=o.ALG_MASK, group_tiles=8)[2]
    assert stm["texel_evals_unique"] <= st["texel_evals_unique"]


# ---------------------------------------------------------------------------
# Fallbacks C and C+ (Sec. 3.4)
# ---------------------------------------------------------------------------
def test_cplus_lane_mapping_eq2(oracle_lib):
    """Eq. 2 with 32 lanes: l = round(31 (c - n) / (31 - n)), computed here in
    exact rationals with halves rounded up; the text's properties: lanes 0
    and 31 are sources whenever two or more lanes remain, a single remaining
    lane maps to 0, and the sources never decrease with c."""
    from fractions import Fraction
    o = oracle_lib
    for n in range(32):
        prev = -1
        for c in range(n, 32):
            got = o.cplus_source(32, n, c)
            if n == 31:
                assert got == 0
                continue
            x = Fraction(31 * (c - n), 31 - n)
            assert got == int(x + Fraction(1, 2)), (n, c)
            assert got >= prev
            prev = got
        if 32 - n >= 2:
            assert o.cplus_source(32, n, n) == 0 and o.cplus_source(32, n, 31) == 31
    assert o.cplus_source(32, 5, 4) == -1 and o.cplus_source(33, 0, 0) == -1


def _fallback_tiles(o, blocks, uv, jac, cov, fallback, alg=None):
    alg = o.ALG_BOX if alg is None else alg
    return o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=alg, seed=9, fallback=fallback, want_tiles=True)


def _tile_lanes(uv, cov, tx, ty):
    """Active lanes of an 8x4 tile with their FP32 setup (texel units)."""
    lanes = []
    for l in range(32):
        px, py = tx * 8 + l % 8, ty * 4 + l // 8
        if not cov[py, px]:
            continue
        xf = np.float32(uv[py, px, 0]) * np.float32(64) - np.float32(0.5)
        yf = np.float32(uv[py, px, 1]) * np.float32(64) - np.float32(0.5)
        ulx, uly = int(np.floor(xf)), int(np.floor(yf))
        s_, t_ = np.float32(xf - np.float32(ulx)), np.float32(yf - np.float32(uly))
        os_, ot_ = np.float32(1) - s_, np.float32(1) - t_
        w = [os_ * ot_, s_ * ot_, os_ * t_, s_ * t_]
        lanes.append((l, px, py, ulx, uly, float(s_), float(t_), w))
    return lanes


def test_fallback_c_is_eq1_in_exact_arithmetic(oracle_lib):
    """Fallback C: every active lane produces its STF texel (the pinned Philox
    draw); each pixel then blends the distinct produced texels of its
    footprint with nonzero weight by eq. 1, evaluated here in exact rationals
    from the pinned block decode: sum w p + (1 - sum w) mean(p), or exact
    bilinear when all of them are present, or the single texel."""
    from fractions import Fraction
    o = oracle_lib
    blocks = synth.random_blocks(64, 64, seed=13)
    uv, jac, cov = _scene_mix(seed=9)
    out, ev, st, tp, _ = _fallback_tiles(o, blocks, uv, jac, cov, o.FALLBACK_C)
    ref_stf = _fallback_tiles(o, blocks, uv, jac, cov, o.FALLBACK_STF)[0]
    bil = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=o.ALG_4TAP)[0]
    tiles_x = 96 // 8
    cases = {"all": 0, "one": 0, "blend": 0}
    for tid in np.nonzero(tp == o.PATH_FALLBACK_BUDGET)[0]:
        ty, tx = divmod(int(tid), tiles_x)
        lanes = _tile_lanes(uv, cov, tx, ty)
        produced = set()
        for (l, px, py, ulx, uly, s_, t_, w) in lanes:
            dx, dy = o.stf_offset(px, py, 0, 9, s_, t_)
            produced.add((ulx + dx, uly + dy))
            assert ev[py, px] == 1
        for (l, px, py, ulx, uly, s_, t_, w) in lanes:
            taps = [(ulx + k % 2, uly + k // 2) for k in range(4)]
            nz = [k for k in range(4) if w[k] > 0]
            pres = [k for k in nz if taps[k] in produced]
            vals = {k: [Fraction(int(v), 255) for v in o.decode_rgba8(blocks, 64, 64, *taps[k])] for k in pres}
            if len(pres) == len(nz):
                cases["all"] += 1
                assert np.array_equal(out[py, px].view(np.uint32), bil[py, px].view(np.uint32))
                continue
            if len(pres) == 1:
                cases["one"] += 1
                assert np.array_equal(out[py, px].view(np.uint32), ref_stf[py, px].view(np.uint32))
                continue
            cases["blend"] += 1
            sw = sum(Fraction(float(w[k])) for k in pres)
            for ch in range(4):
                sp = sum(vals[k][ch] for k in pres)
                exact = sum(Fraction(float(w[k])) * vals[k][ch] for k in pres) + (1 - sw) * sp / len(pres)
                assert abs(float(exact) - float(out[py, px, ch])) <= 4e-7 * max(1.0, abs(float(exact))), (tid, l, ch)
    assert min(cases.values()) > 10, cases


def test_fallback_cplus_invariants(oracle_lib):
    """Fallback C+: the distinct STF texels are produced by the first n
    active lanes and the other lanes add texels outside that set, so every
    pixel sees at least the texels of fallback C: where C is exact bilinear
    so is C+.  Quality improves as Sec. 3.4 states: mean absolute error
    against bilinear over the fallback tiles, C+ < C < one-tap STF."""
    o = oracle_lib
    blocks = synth.random_blocks(64, 64, seed=13)
    uv, jac, cov = _scene_mix(seed=9)
    bil = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=o.ALG_4TAP)[0]
    res = {f: _fallback_tiles(o, blocks, uv, jac, cov, f) for f in (o.FALLBACK_STF, o.FALLBACK_C, o.FALLBACK_CPLUS)}
    outp, evp, stp, tpp, _ = res[o.FALLBACK_CPLUS]
    outc = res[o.FALLBACK_C][0]
    tiles_x = 96 // 8
    mask = np.zeros(cov.shape, bool)
    for tid in np.nonzero(tpp == o.PATH_FALLBACK_BUDGET)[0]:
        ty, tx = divmod(int(tid), tiles_x)
        lanes = _tile_lanes(uv, cov, tx, ty)
        stf = []
        for (l, px, py, ulx, uly, s_, t_, w) in lanes:
            dx, dy = o.stf_offset(px, py, 0, 9, s_, t_)
            stf.append((ulx + dx, uly + dy))
            mask[py, px] = True
        n = len(set(stf))
        counts = [int(evp[py, px]) for (l, px, py, *_r) in lanes]
        assert counts[:n] == [1] * n and all(c in (0, 1) for c in counts[n:])
        for (l, px, py, ulx, uly, s_, t_, w) in lanes:
            taps = [(ulx + k % 2, uly + k // 2) for k in range(4)]
            if all(taps[k] in set(stf) for k in range(4) if w[k] > 0):
                # C has every texel of this footprint, hence so has C+: both exact bilinear
                assert np.array_equal(outc[py, px].view(np.uint32), bil[py, px].view(np.uint32))
                assert np.array_equal(outp[py, px].view(np.uint32), bil[py, px].view(np.uint32))
    assert mask.sum() > 100
    err = {f: float(np.abs(r[0][mask] - bil[mask]).mean()) for f, r in res.items()}
    assert err[o.FALLBACK_CPLUS] < err[o.FALLBACK_C] < err[o.FALLBACK_STF], err
    # outside the fallback tiles nothing changes
    np.testing.assert_array_equal(outp[~mask], res[o.FALLBACK_STF][0][~mask])


def test_mask11_equals_mask16_when_bbox_fits(oracle_lib):
    o = oracle_lib
    blocks = synth.random_blocks(64, 64, seed=14)
    uv, jac, cov = _scene_mix(seed=21)
    a16 = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=o.ALG_MASK, mask_dim=16, want_tiles=True)
    a11 = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=o.ALG_MASK, mask_dim=11, want_tiles=True)
    fits11 = a11[4] >= 0
    np.testing.assert_array_equal(a16[4][fits11], a11[4][fits11])
    np.testing.assert_array_equal(a16[3][fits11], a11[3][fits11])
    # on this magnified scene the two masks agree everywhere (Sec. 3.3: identical results)
    np.testing.assert_array_equal(a16[0], a11[0])


def test_edge_remapping(oracle_lib):
    """Supplemental Sec. 2: with remapping a wave succeeds when popcount(A) >= n;
    without it the first n lanes must be active."""
    o = oracle_lib
    blocks = synth.random_blocks(64, 64, seed=15)
    # one tile at magnification 4: the 8x4 footprint needs 3x2 = 6 texels (Box)
    W, H = 8, 4
    ly, lx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    uv = np.stack([(lx / 4 + 30.3) / 64, (ly / 4 + 30.6) / 64], -1).astype(np.float32)
    jac = np.tile(np.array([0.25 / 64, 0, 0, 0.25 / 64], np.float32), (H, W, 1))
    cov = np.ones((H, W), np.uint8)
    cov[0, 0:3] = 0  # lanes 0..2 inactive
    _, _, _, tp, tn = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=o.ALG_BOX, want_tiles=True, edge_remap=1)
    n = int(tn[0])
    assert 2 <= n <= 29 and tp[0] == o.PATH_SUCCESS
    _, _, _, tp0, _ = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=o.ALG_BOX, want_tiles=True, edge_remap=0)
    assert tp0[0] == o.PATH_FALLBACK_BUDGET
    # only two active lanes but n > 2 -> fallback even with remapping
    cov2 = np.zeros((H, W), np.uint8)
    cov2[2, 3] = cov2[3, 7] = 1
    _, ev, _, tp2, tn2 = o.filter_frame(blocks, 64, 64, uv, jac, cov2, alg=o.ALG_MASK, want_tiles=True)
    assert tn2[0] > 2 and tp2[0] == o.PATH_FALLBACK_BUDGET and ev.sum() == 2


# ---------------------------------------------------------------------------
# Thresholds of Fig. 4 and the 54-texel maximum of Sec. 5 (brute force)
# ---------------------------------------------------------------------------
def _sweep(o, m, alg, n_phase, degrees=np.arange(0, 91, 1.0)):
    sc = synth.rotated_quad_tiles(m, degrees, n_phase)
    blocks = synth.random_blocks(4096, 4096, seed=16) if not hasattr(_sweep, "blocks") else _sweep.blocks
    _sweep.blocks = blocks
    _, _, st, tp, tn = o.filter_frame(blocks, 4096, 4096, sc.uv, sc.jac, None, alg=alg, want_tiles=True)
    return tp, tn


@pytest.mark.slow
def test_fig4_thresholds_and_max_unique(oracle_lib):
    o = oracle_lib
    vals = {r[1]: float(r[2]) for r in _read_lines("paper_values.txt") if r[0] == "threshold"}
    max_unique = int([r for r in _read_lines("paper_values.txt") if r[0] == "max_unique_m1"][0][1])
    nph = 400
    for name, alg in (("list_merge", o.ALG_LIST_MERGE), ("mask", o.ALG_MASK), ("box", o.ALG_BOX)):
        thr = vals[name]
        tp, _ = _sweep(o, thr + 0.01, alg, nph)
        assert np.all(tp == o.PATH_SUCCESS), name
        tp, _ = _sweep(o, thr - 0.05, alg, nph)
        assert np.any(tp == o.PATH_FALLBACK_BUDGET), name
    # worst Box case sits at 45 degrees
    tp45, _ = _sweep(o, vals["box"] - 0.02, o.ALG_BOX, 1000, degrees=[45.0])
    tp0, _ = _sweep(o, vals["box"] - 0.02, o.ALG_BOX, 1000, degrees=[0.0])
    assert np.any(tp45 != o.PATH_SUCCESS) and np.all(tp0 == o.PATH_SUCCESS)
    # at magnification 1.0 the most unique texels any 8x4 wave needs
    _, tn = _sweep(o, 1.0, o.ALG_LIST_MERGE, 300, degrees=np.arange(0, 91, 1.0))
    assert int(tn.max()) == max_unique


def test_two_texels_per_lane_always_succeed_at_unit_magnification(oracle_lib):
    """Sec. 5: an 8x4 wave needs at most 54 distinct texels at magnification
    1, so two texel evaluations per lane always succeed once every pixel is
    magnified.  With texels_per_lane 2 and budget 64, List Merge and the
    16x16 mask succeed on every rotation and phase just above magnification
    1, the outputs equal per-pixel bilinear bitwise, and the counts follow
    the round-robin assignment: active lane a produces texels a and a + 32."""
    o = oracle_lib
    degrees = np.arange(0, 91, 3.0)
    sc = synth.rotated_quad_tiles(1.001, degrees, 60)
    blocks = synth.random_blocks(4096, 4096, seed=16)
    ref = o.filter_frame(blocks, 4096, 4096, sc.uv, sc.jac, None, alg=o.ALG_4TAP)[0]
    for alg, md in ((o.ALG_LIST_MERGE, 16), (o.ALG_MASK, 16)):
        out1, ev1, st1, tp1, tn1 = o.filter_frame(blocks, 4096, 4096, sc.uv, sc.jac, None, alg=alg, mask_dim=md,
                                                  want_tiles=True)
        assert np.any(tp1 == o.PATH_FALLBACK_BUDGET)  # one texel per lane is not enough here
        out, ev, st, tp, tn = o.filter_frame(blocks, 4096, 4096, sc.uv, sc.jac, None, alg=alg, mask_dim=md,
                                             budget=64, texels_per_lane=2, want_tiles=True)
        assert np.all(tp == o.PATH_SUCCESS) and tn.max() > 32
        assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))
        for tid in range(tp.size):
            n = int(tn[tid])
            cnt = ev[tid * 4:tid * 4 + 4].ravel()
            expect = np.array([(a < n) + (a + 32 < n) for a in range(32)], np.uint8)
            np.testing.assert_array_equal(cnt, expect)
        # tiles that one texel per lane already handled are unchanged
        same = tp1 == o.PATH_SUCCESS
        rows = np.repeat(same, 4)
        np.testing.assert_array_equal(ev[rows], ev1[rows])


# ---------------------------------------------------------------------------
# One-tap STF: unbiased for bilinear (Sec. 3.4 opening; Pharr et al. 2024)
# ---------------------------------------------------------------------------
def test_stf_mean_converges_to_bilinear(oracle_lib):
    o = oracle_lib
    Wt = Ht = 16
    blocks = synth.random_blocks(Wt, Ht, seed=17)
    g = np.random.default_rng(8)
    W, H = 8, 4
    uv = g.uniform(0.1, 0.9, (H, W, 2)).astype(np.float32)
    jac = np.zeros((H, W, 4), np.float32)
    ref, _, _ = o.filter_frame(blocks, Wt, Ht, uv, jac, alg=o.ALG_4TAP)
    S = 4096
    acc = np.zeros_like(ref, dtype=np.float64)
    acc2 = np.zeros_like(acc)
    for seed in range(S):
        out, ev, _ = o.filter_frame(blocks, Wt, Ht, uv, jac, alg=o.ALG_STF, seed=seed * 0x9E3779B97F4A7C15 % 2**64)
        assert np.all(ev == 1)
        acc += out
        acc2 += out.astype(np.float64) ** 2
    mean = acc / S
    var = np.maximum(acc2 / S - mean ** 2, 0)
    bound = 4.5 * np.sqrt(var / S) + 2.0 ** -22
    assert np.all(np.abs(mean - ref) <= bound)


@pytest.mark.parametrize("flt", ["bspline", "catmull_rom"])
def test_bicubic_stf_mean_converges(oracle_lib, flt):
    """One-tap STF for the bicubic filters draws a tap per axis with
    probability |w| / sum |w|; the B-spline returns the texel and Catmull-Rom
    the texel times the signed sums, so the mean over seeds converges to the
    filter, negative lobes included."""
    o = oracle_lib
    f = {"bspline": o.FILTER_BSPLINE, "catmull_rom": o.FILTER_CATMULL_ROM}[flt]
    Wt = Ht = 16
    blocks = synth.random_blocks(Wt, Ht, seed=19)
    g = np.random.default_rng(6)
    W, H = 8, 4
    uv = g.uniform(0.2, 0.8, (H, W, 2)).astype(np.float32)
    jac = np.zeros((H, W, 4), np.float32)
    ref, _, _ = o.filter_frame(blocks, Wt, Ht, uv, jac, alg=o.ALG_4TAP, filter=f)
    S = 4096
    acc = np.zeros_like(ref, dtype=np.float64)
    acc2 = np.zeros_like(acc)
    for seed in range(S):
        out, ev, _ = o.filter_frame(blocks, Wt, Ht, uv, jac, alg=o.ALG_STF, filter=f,
                                    seed=seed * 0x9E3779B97F4A7C15 % 2**64)
        assert np.all(ev == 1)
        acc += out
        acc2 += out.astype(np.float64) ** 2
    mean = acc / S
    var = np.maximum(acc2 / S - mean ** 2, 0)
    assert np.all(np.abs(mean - ref) <= 4.5 * np.sqrt(var / S) + 2.0 ** -20)


@pytest.mark.parametrize("flt", ["bspline", "catmull_rom"])
def test_bicubic_success_reproduces_per_pixel_bitwise(oracle_lib, flt):
    """Sec. 4.2: the same algorithms serve any discrete filter; a bicubic
    success tile equals the per-pixel 16-tap filter bitwise, Mask-16 and List
    Merge agree on n whenever the box fits, and the first n active lanes
    count 1."""
    o = oracle_lib
    f = {"bspline": o.FILTER_BSPLINE, "catmull_rom": o.FILTER_CATMULL_ROM}[flt]
    blocks = synth.random_blocks(64, 64, seed=13)
    uv, jac, cov = _scene_mix(seed=4)
    ref = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=o.ALG_4TAP, filter=f)[0]
    res = {}
    for name, a in (("box", o.ALG_BOX), ("mask", o.ALG_MASK), ("list", o.ALG_LIST_MERGE)):
        out, ev, st, tp, tn = o.filter_frame(blocks, 64, 64, uv, jac, cov, alg=a, filter=f, want_tiles=True)
        res[name] = (tp, tn)
        tiles_x = 96 // 8
        succ = np.nonzero(tp == o.PATH_SUCCESS)[0]
        assert succ.size > 10, name
        for tid in succ:
            ty, tx = divmod(int(tid), tiles_x)
            sl = (slice(ty * 4, ty * 4 + 4), slice(tx * 8, tx * 8 + 8))
            assert np.array_equal(out[sl].view(np.uint32), ref[sl].view(np.uint32))
            act = cov[sl].ravel() != 0
            expect = np.zeros(32, np.uint8)
            expect[np.nonzero(act)[0][:int(tn[tid])]] = 1
            np.testing.assert_array_equal(ev[sl].ravel(), expect)
    fit = res["mask"][1] >= 0
    np.testing.assert_array_equal(res["mask"][1][fit], res["list"][1][fit])


def test_stf_choice_frequencies_equal_weights(oracle_lib):
    """The separable choice picks tap (dx,dy) with probability equal to its
    bilinear weight: compare frequencies over 20000 counters with a 5-sigma bound."""
    o = oracle_lib
    s, t = np.float32(0.3), np.float32(0.8)
    n = 20000
    counts = np.zeros((2, 2))
    for i in range(n):
        dx, dy = o.stf_offset(i % 200, i // 200, 7, 12345, s, t)
        counts[dy, dx] += 1
    p = np.array([[(1 - s) * (1 - t), s * (1 - t)], [(1 - s) * t, s * t]])
    sigma = np.sqrt(p * (1 - p) / n)
    assert np.all(np.abs(counts / n - p) <= 5 * sigma)


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------
def test_edge_cases(oracle_lib):
    o = oracle_lib
    blocks = synth.random_blocks(16, 16, seed=18)
    # empty frame
    out, ev, st = o.filter_frame(blocks, 16, 16, np.zeros((0, 5, 2), np.float32), np.zeros((0, 5, 4), np.float32))
    assert out.shape == (0, 5, 4) and st["tiles_total"] == 0
    # ragged frame: 13 x 7 with every kind of inactive pixel
    g = np.random.default_rng(2)
    uv = g.uniform(0.0, 1.0, (7, 13, 2)).astype(np.float32)
    uv[0, 0] = np.nan
    uv[1, 1] = [1e9, 0.5]
    jac = np.tile(np.array([0.01 / 16, 0, 0, 0.01 / 16], np.float32), (7, 13, 1))
    cov = np.ones((7, 13), np.uint8)
    cov[2, 2] = 0
    for alg in range(5):
        out, ev, st = o.filter_frame(blocks, 16, 16, uv, jac, cov, alg=alg)
        assert st["pixels_active"] == 13 * 7 - 3
        for (y, x) in ((0, 0), (1, 1), (2, 2)):
            assert ev[y, x] == 0 and np.all(out[y, x] == 0)
        assert st["tiles_total"] == 2 * 2
    # bad arguments
    with pytest.raises(ValueError):
        o.filter_frame(blocks, 16, 16, uv, jac, tile_w=4, tile_h=4)
    with pytest.raises(ValueError):
        o.filter_frame(blocks, 16, 16, uv, jac, alg=o.ALG_MASK, mask_dim=12)


# ---------------------------------------------------------------------------
# Bands of a view
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("alg,fallback", [(2, 0), (3, 0), (4, 0), (4, 2)])
def test_band_equals_rows_of_the_whole_view(oracle_lib, alg, fallback):
    """A band of whole tile rows filtered on its own with y_offset gives the
    same pixels and counts as those rows of the whole view (the offset enters
    only the per-pixel STF counters; the scene has minified and over-budget
    tiles, so the stochastic draws are exercised), and it is refused when it
    would split tile rows."""
    Wt = Ht = 256
    blocks = synth.random_blocks(Wt, Ht, seed=5)
    sc = synth.ground_plane_with_quads(160, 96, Wt, Ht)
    kw = dict(alg=alg, seed=77, view=3, mask_dim=11, fallback=fallback)
    full, full_ev, st = oracle_lib.filter_frame(blocks, Wt, Ht, sc.uv, sc.jac, sc.coverage, **kw)
    assert st["tiles_fallback_minified"] > 0 and st["tiles_success"] > 0
    y0, y1 = 40, 72
    band, band_ev, _ = oracle_lib.filter_frame(blocks, Wt, Ht, sc.uv[y0:y1], sc.jac[y0:y1], sc.coverage[y0:y1],
                                              y_offset=y0, **kw)
    assert np.array_equal(band.view(np.uint32), full[y0:y1].view(np.uint32))
    assert np.array_equal(band_ev, full_ev[y0:y1])
    # without the offset the STF draws of the band are those of other pixels
    moved, _, _ = oracle_lib.filter_frame(blocks, Wt, Ht, sc.uv[y0:y1], sc.jac[y0:y1], sc.coverage[y0:y1], **kw)
    assert not np.array_equal(moved.view(np.uint32), full[y0:y1].view(np.uint32))
    with pytest.raises(ValueError):
        oracle_lib.filter_frame(blocks, Wt, Ht, sc.uv[y0 + 2:y1], sc.jac[y0 + 2:y1], sc.coverage[y0 + 2:y1],
                                y_offset=y0 + 2, **kw)
