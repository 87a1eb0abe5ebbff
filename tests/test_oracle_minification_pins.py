"""Pins of the oracle's minification vote (step a2) against hand-derived flags.

The rule being pinned (Sec. 4: tiles with minified pixels leave the
collaborative path; the magnification m of a pixel is 1/rho, rho the larger
column norm of its UV Jacobian measured in texels per pixel):

    rho_x^2 = (du/dx * Wt)^2 + (dv/dx * Ht)^2,  rho_y^2 = (du/dy * Wt)^2 + (dv/dy * Ht)^2
    a pixel is minified iff rho_x^2 > 1 or rho_y^2 > 1 (a NaN counts as minified)
    a tile leaves for one-tap STF iff at least one ACTIVE pixel is minified.

Every expected flag below is written by hand from that definition, with the
derivation beside it, never computed by re-running a formula.  The Jacobians
are given in texels per pixel, T = (a, b, c, d) = (du/dx*Wt, dv/dx*Ht,
du/dy*Wt, dv/dy*Ht), and passed in UV units as (a/Wt, b/Ht, c/Wt, d/Ht).
Wt and Ht are unequal powers of two and the entries are short dyadic
fractions, so the division and the oracle's multiplication back are exact and
only the squares and the sum can round.

A single 8x4 tile is filtered: every pixel samples the same point, so the
footprint is one 2x2 texel square (n = 4 <= 32) and the tile succeeds unless
the vote sends it to STF.  The pixel under test is one lane; every other
active lane has a zero Jacobian (rho = 0, magnified).  The tile's path and
per-pixel counts reveal the vote:
    success   -> path SUCCESS, the 4 texels counted once each (sum 4);
    minified  -> path FALLBACK_MINIFIED, every active pixel counts 1.
Plausible mistakes each fail a case here: row norms instead of column norms
(the transposed pair), a missing or swapped Wt/Ht factor (the unequal sizes),
`<` instead of `<=` at rho = 1, a vote in double precision instead of FP32
(the rounding case), a per-lane instead of per-tile decision, and a vote
taken over inactive lanes.
"""
import numpy as np
import pytest

from paper_2506_17770_gb300 import synth

WT, HT = 64, 32           # unequal, so a dropped or swapped scale factor shows
TW, TH = 8, 4
U0 = (10 + 0.5 + 0.25) / WT   # texel-space x = 10.25 after the -0.5 shift: exact
V0 = (7 + 0.5 + 0.25) / HT    # texel-space y = 7.25


def _frame(T_lane, lane=17, inactive=False, tile_w=TW, tile_h=TH):
    """One tile; lane `lane` gets texel-space Jacobian T_lane, others zero."""
    uv = np.empty((tile_h, tile_w, 2), np.float32)
    uv[..., 0] = U0
    uv[..., 1] = V0
    jac = np.zeros((tile_h, tile_w, 4), np.float32)
    a, b, c, d = T_lane
    ly, lx = divmod(lane, tile_w)
    jac[ly, lx] = np.array([np.float32(a) / np.float32(WT), np.float32(b) / np.float32(HT),
                            np.float32(c) / np.float32(WT), np.float32(d) / np.float32(HT)], np.float32)
    cov = None
    if inactive:
        cov = np.ones((tile_h, tile_w), np.uint8)
        cov[ly, lx] = 0
    return uv, jac, cov


def _vote(oracle_lib, T_lane, alg, lane=17, inactive=False, tile_w=TW, tile_h=TH):
    blocks = synth.random_blocks(WT, HT)
    uv, jac, cov = _frame(T_lane, lane, inactive, tile_w, tile_h)
    _, ev, st, tp, tn = oracle_lib.filter_frame(blocks, WT, HT, uv, jac, cov, alg=alg, tile_w=tile_w,
                                                tile_h=tile_h, want_tiles=True)
    return int(tp[0]), ev, st


ALGS = [2, 3, 4]  # List Merge, Box, Mask: the vote is shared by all three

# (name, T in texels per pixel, minified?) -- each flag derived by hand:
CASES = [
    # isotropic, rho = 1 - 2^-20: rho^2 = 1 - 2^-19 + 2^-40, RN in FP32 -> 1 - 2^-19 <= 1
    ("iso_below_1", (1 - 2.0**-20, 0.0, 0.0, 1 - 2.0**-20), False),
    # isotropic, rho = 1 exactly: rho^2 = 1, and 1 <= 1 -> magnified (m = 1 is magnification)
    ("iso_exactly_1", (1.0, 0.0, 0.0, 1.0), False),
    # isotropic, rho = 1 + 2^-20: rho^2 rounds to 1 + 2^-19 > 1 -> minified
    ("iso_above_1", (1 + 2.0**-20, 0.0, 0.0, 1 + 2.0**-20), True),
    # the axes swapped (du/dy, dv/dx carry the scale): columns (0,1), (1,0), norms 1 -> magnified
    ("swap_exactly_1", (0.0, 1.0, 1.0, 0.0), False),
    # anisotropic: x column (3/2, 0) norm^2 9/4 > 1 even though y column (0, 1/2) is 1/4
    ("aniso_x_column_over", (1.5, 0.0, 0.0, 0.5), True),
    # anisotropic: only the y column (0, 5/4) is over, 25/16 > 1
    ("aniso_y_column_over", (0.5, 0.0, 0.0, 1.25), True),
    # column norms: x column (13/16, 13/16) -> 338/256 > 1 -> minified; its row norms are
    # (13/16, 0) -> 169/256 and (13/16, 1/8) -> 173/256, both <= 1: a row-norm vote says magnified
    ("columns_not_rows", (0.8125, 0.8125, 0.0, 0.125), True),
    # the transpose of the previous: columns (13/16, 0) and (13/16, 1/8) -> 169/256 and
    # 173/256, both <= 1 -> magnified; its rows give 338/256 > 1, so a row-norm vote says minified
    ("columns_not_rows_transposed", (0.8125, 0.0, 0.8125, 0.125), False),
    # Wt != Ht: dv/dx alone, 5/4 texels -> 25/16 > 1 -> minified.  With Ht dropped
    # (dv/dx * 1) the norm is tiny; with Wt in place of Ht it is 5/2 -> still over
    ("dv_dx_needs_Ht", (0.0, 1.25, 0.0, 0.0), True),
    # (5/8, 5/8) in texels -> 50/64 <= 1 -> magnified.  With Wt in place of Ht the
    # v term is (5/8 * 64/32)^2 = 25/16 and the pixel would read as minified
    ("du_dv_scaled_separately", (0.625, 0.625, 0.0, 0.0), False),
    # y column the same way: (5/8, 5/8) -> 50/64 -> magnified
    ("y_column_scaled_separately", (0.0, 0.0, 0.625, 0.625), False),
    # negative entries square to the same norms: (-3/4, -3/4) -> 18/16 > 1 -> minified
    ("negative_entries", (-0.75, -0.75, 0.0, 0.0), True),
    # the vote is taken in FP32 with round-to-nearest: (1, 2^-13) has rho^2 = 1 + 2^-26
    # exactly, which is > 1 in exact arithmetic, but 1 + 2^-26 rounds to 1.0f (half an ulp
    # of 1 is 2^-24) and 1.0f <= 1 -> magnified.  A vote in double would say minified
    ("fp32_rounding_at_1", (1.0, 2.0**-13, 0.0, 0.0), False),
    # 2^-12 instead: 1 + 2^-24 is a tie, and round-to-nearest-even keeps 1.0f -> magnified
    ("fp32_tie_at_1", (1.0, 2.0**-12, 0.0, 0.0), False),
    # 2^-11: 1 + 2^-22 is representable and > 1 -> minified
    ("fp32_just_over_1", (1.0, 2.0**-11, 0.0, 0.0), True),
    # non-finite derivatives: a NaN gives NaN norms; the pixel counts as minified
    ("nan_du_dx", (float("nan"), 0.0, 0.0, 0.0), True),
    ("nan_dv_dy", (0.0, 0.0, 0.0, float("nan")), True),
    # an infinite derivative has an infinite norm -> minified
    ("inf_du_dy", (0.0, 0.0, float("inf"), 0.0), True),
    ("minus_inf_dv_dx", (0.0, float("-inf"), 0.0, 0.0), True),
    # a finite derivative whose square overflows FP32 (2^70 texels) -> +inf -> minified
    ("square_overflows", (2.0**70, 0.0, 0.0, 0.0), True),
]


@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("name,T,minified", CASES, ids=[c[0] for c in CASES])
def test_minification_flag(oracle_lib, alg, name, T, minified):
    path, ev, st = _vote(oracle_lib, T, alg)
    if minified:
        assert path == oracle_lib.PATH_FALLBACK_MINIFIED, name
        assert st["tiles_fallback_minified"] == 1
        # one-tap STF for the whole tile: every pixel, minified or not, counts 1
        assert np.all(ev == 1), name
        assert st["texel_evals"] == TW * TH
    else:
        assert path == oracle_lib.PATH_SUCCESS, name
        assert st["tiles_success"] == 1
        # the tile's 2x2 footprint, each texel produced once
        assert int(ev.sum()) == 4 and st["texel_evals"] == 4, name


@pytest.mark.parametrize("rho,minified", [(0.9375, False), (1.0625, True)])
@pytest.mark.parametrize("theta", [0.3, 1.0, 2.0, 4.0, 5.5])
def test_rotated_jacobian(oracle_lib, rho, theta, minified):
    """A rotation scaled by rho has both column norms equal to rho whatever the
    angle: 15/16 -> rho^2 = 0.879 (magnified), 17/16 -> 1.129 (minified); the
    FP32 rounding of cos/sin moves rho^2 by ~1e-7, far from 1."""
    c, s = np.cos(theta), np.sin(theta)
    T = (rho * c, rho * s, -rho * s, rho * c)
    path, ev, _ = _vote(oracle_lib, T, 3)
    assert path == (oracle_lib.PATH_FALLBACK_MINIFIED if minified else oracle_lib.PATH_SUCCESS)


@pytest.mark.parametrize("lane", [0, 17, 31])
@pytest.mark.parametrize("alg", ALGS)
def test_one_minified_lane_sends_the_whole_tile(oracle_lib, lane, alg):
    """Per-tile, not per-lane: one minified active pixel (rho_x^2 = 4) sends
    all 32 to one-tap STF; the 31 magnified pixels count 1, not 0 or 4."""
    path, ev, st = _vote(oracle_lib, (2.0, 0.0, 0.0, 0.0), alg, lane=lane)
    assert path == oracle_lib.PATH_FALLBACK_MINIFIED
    assert np.all(ev == 1) and st["pixels_active"] == 32


@pytest.mark.parametrize("lane", [0, 17, 31])
@pytest.mark.parametrize("alg", ALGS)
def test_inactive_minified_lane_does_not_vote(oracle_lib, lane, alg):
    """The same minified Jacobian on a pixel with coverage 0: only active
    pixels vote, so the tile succeeds with the other 31 (count sum 4)."""
    path, ev, st = _vote(oracle_lib, (2.0, 0.0, 0.0, 0.0), alg, lane=lane, inactive=True)
    assert path == oracle_lib.PATH_SUCCESS
    assert st["pixels_active"] == 31
    ly, lx = divmod(lane, TW)
    assert ev[ly, lx] == 0 and int(ev.sum()) == 4


@pytest.mark.parametrize("shape", [(4, 8), (16, 2)])
def test_vote_with_other_tile_shapes(oracle_lib, shape):
    """Row-major lanes in 4x8 and 16x2 tiles: the last lane's pixel is the
    bottom-right one, and its minified Jacobian decides the tile alone."""
    tw, th = shape
    path, ev, _ = _vote(oracle_lib, (0.0, 0.0, 0.0, 1.5), 4, lane=31, tile_w=tw, tile_h=th)
    assert path == oracle_lib.PATH_FALLBACK_MINIFIED and np.all(ev == 1)
    path, ev, _ = _vote(oracle_lib, (0.0, 0.0, 0.0, 1.0), 4, lane=31, tile_w=tw, tile_h=th)
    assert path == oracle_lib.PATH_SUCCESS and int(ev.sum()) == 4
