"""CPU oracle for Collaborative Texture Filtering (arXiv 2506.17770).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / ``--impl reference`` leg of ``bench.py`` import this package.  The
product package ``paper_2506_17770_gb300`` never imports it, and the two share no
code: the oracle is plain C (``ctf_oracle.c``, ``ctf_oracle_mlp.c``) compiled with
gcc and called through ctypes with numpy arrays.

Each function cites the passage of the paper it restates; see the C sources.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "ctf_oracle.c"), os.path.join(_HERE, "ctf_oracle_mlp.c")]
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ALG_4TAP, ALG_STF, ALG_LIST_MERGE, ALG_BOX, ALG_MASK = 0, 1, 2, 3, 4
PATH_EMPTY, PATH_SUCCESS, PATH_FALLBACK_BUDGET, PATH_FALLBACK_MINIFIED, PATH_DIRECT = 0, 1, 2, 3, 4
FALLBACK_STF, FALLBACK_C, FALLBACK_CPLUS = 0, 1, 2
FILTER_BILINEAR, FILTER_BSPLINE, FILTER_CATMULL_ROM = 0, 1, 2
STAT_NAMES = ("tiles_total", "tiles_empty", "tiles_direct", "tiles_success",
              "tiles_fallback_budget", "tiles_fallback_minified", "pixels_active", "texel_evals",
              "texel_evals_unique")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    stale = force or not os.path.exists(_SO) or any(
        os.path.getmtime(s) > os.path.getmtime(_SO) for s in _SRCS)
    if stale:
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp] + _SRCS + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i32, u64 = ctypes.c_int, ctypes.c_uint64
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_philox4x64_10.argtypes = [P, P, P]
            lib.oracle_h.argtypes = [P, i32, i32]
            lib.oracle_h.restype = i32
            lib.oracle_hinv.argtypes = [P, i32, i32]
            lib.oracle_hinv.restype = i32
            lib.oracle_decode_rgba8.argtypes = [P, i32, i32, i32, i32, P]
            lib.oracle_stf_offset.argtypes = [i32, i32, i32, u64, ctypes.c_float, ctypes.c_float, P, P]
            lib.oracle_filter.argtypes = [P, i32, i32, P, P, P, i32, i32, i32, i32, u64, i32, i32, i32,
                                          i32, i32, i32, i32, i32, i32, i32, P, P, P, P, P]
            lib.oracle_filter.restype = i32
            lib.oracle_cplus_source.argtypes = [i32, i32, i32]
            lib.oracle_cplus_source.restype = i32
            lib.oracle_filter_learned_f64.argtypes = [P, i32, i32, P, P, P, i32, i32, i32, i32, u64, i32,
                                                      i32, i32, i32, i32, i32, i32, i32, i32, i32, P, P, P, P,
                                                      P]
            lib.oracle_filter_learned_f64.restype = i32
            lib.oracle_mlp_features_f64.argtypes = [P, i32, i32, i32, i32, P]
            lib.oracle_mlp_texel_f64.argtypes = [P, i32, i32, i32, i32, P]
            lib.oracle_mlp_decode_f64.argtypes = [P, i32, i32, i32, P, P, P]
            lib.oracle_mlp_loss_grad_f64.argtypes = [P, i32, i32, i32, P, P, P] + [P] * 8
            lib.oracle_mlp_loss_grad_f64.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# Philox, bijection, block decode
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox4x64_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint64).copy()
    k = np.asarray(key, dtype=np.uint64).copy()
    out = np.zeros(4, np.uint64)
    _load().oracle_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def _words(B: int, nwords: int):
    return np.array([(B >> (32 * w)) & 0xFFFFFFFF for w in range(nwords)], dtype=np.uint32)


def h(i: int, B: int, nwords: int = 8) -> int:
    """h(i, B): position of the i-th set bit (Sec. 3.3, Fig. 3)."""
    return _load().oracle_h(_ptr(_words(B, nwords)), nwords, i)


def hinv(t: int, B: int, nwords: int = 8) -> int:
    """h^-1(t, B): number of set bits of B below position t (Sec. 3.3)."""
    return _load().oracle_hinv(_ptr(_words(B, nwords)), nwords, t)


def decode_rgba8(blocks: np.ndarray, Wt: int, Ht: int, x: int, y: int) -> np.ndarray:
    b = np.ascontiguousarray(blocks, dtype=np.uint8)
    out = np.zeros(4, np.uint8)
    _load().oracle_decode_rgba8(_ptr(b), Wt, Ht, x, y, _ptr(out))
    return out


def cplus_source(na, n, c):
    """Eq. 2 lane mapping of fallback C+ over na active lanes (-1 if out of range)."""
    return int(_load().oracle_cplus_source(na, n, c))


def stf_offset(px, py, view, seed, s, t):
    dx, dy = ctypes.c_int(), ctypes.c_int()
    _load().oracle_stf_offset(px, py, view, seed, s, t, ctypes.byref(dx), ctypes.byref(dy))
    return dx.value, dy.value


# ---------------------------------------------------------------------------
# Full-frame filter
# ---------------------------------------------------------------------------
def filter_frame(blocks, Wt, Ht, uv, jac, coverage=None, *, view=0, alg=ALG_BOX, seed=0,
                 tile_w=8, tile_h=4, budget=32, mask_dim=16, edge_remap=1, group_tiles=0, fallback=0,
                 texels_per_lane=1, filter=0, y_offset=0, want_tiles=False):
    """Filter one W x H frame with the exact block decode (FP32 arithmetic).

    fallback: 0 one-tap STF, 1 fallback C, 2 fallback C+ for over-budget tiles.
    y_offset: the frame is the band of a larger view that starts at this row
    (a multiple of tile_h); it enters only the per-pixel STF counters.
    group_tiles > 0: stats["texel_evals_unique"] counts the distinct clamped
    texels evaluated per group of that many consecutive tiles.
    Returns (rgba[H,W,4] float32, evals[H,W] uint8, stats dict[, tile_path, tile_n]).
    """
    uv = np.ascontiguousarray(uv, dtype=np.float32)
    jac = np.ascontiguousarray(jac, dtype=np.float32)
    H, W = uv.shape[0], uv.shape[1]
    assert uv.shape == (H, W, 2) and jac.shape == (H, W, 4)
    cov = None if coverage is None else np.ascontiguousarray(coverage, dtype=np.uint8)
    b = np.ascontiguousarray(blocks, dtype=np.uint8)
    out = np.zeros((H, W, 4), np.float32)
    ev = np.zeros((H, W), np.uint8)
    ntiles = ((W + tile_w - 1) // tile_w) * ((H + tile_h - 1) // tile_h) if W and H else 0
    tp = np.zeros(max(ntiles, 1), np.int32)
    tn = np.zeros(max(ntiles, 1), np.int32)
    stats = np.zeros(9, np.int64)
    rc = _load().oracle_filter(_ptr(b), Wt, Ht, _ptr(uv), _ptr(jac), _ptr(cov), W, H, view, alg, seed,
                               tile_w, tile_h, budget, mask_dim, edge_remap, group_tiles, fallback,
                               texels_per_lane, filter, y_offset, _ptr(out),
                               _ptr(ev),
                               _ptr(tp), _ptr(tn), _ptr(stats))
    if rc != 0:
        raise ValueError(f"oracle_filter rejected its arguments (rc={rc})")
    sd = dict(zip(STAT_NAMES, (int(v) for v in stats)))
    if want_tiles:
        return out, ev, sd, tp[:ntiles], tn[:ntiles]
    return out, ev, sd


# ---------------------------------------------------------------------------
# Learned decode (FP64)
# ---------------------------------------------------------------------------
class _MLPStruct(ctypes.Structure):
    _fields_ = [("ch", ctypes.c_int), ("gw", ctypes.c_int * 2), ("gh", ctypes.c_int * 2),
                ("latent", ctypes.c_void_p * 2), ("nin", ctypes.c_int), ("hidden", ctypes.c_int),
                ("nout", ctypes.c_int), ("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p),
                ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p), ("w3", ctypes.c_void_p),
                ("b3", ctypes.c_void_p), ("saturate", ctypes.c_int)]


class MLP:
    """FP64 learned-decode parameters.  ``latents`` is a pair of [gh, gw, ch]
    arrays; w1 [hidden, 2ch], w2 [hidden, hidden], w3 [nout, hidden]; biases
    1-D.  Values are converted to float64 exactly (FP16/E4M3 are subsets)."""

    def __init__(self, latents, w1, b1, w2, b2, w3, b3, saturate=True):
        self._keep = [np.ascontiguousarray(np.asarray(a, dtype=np.float64))
                      for a in (latents[0], latents[1], w1, b1, w2, b2, w3, b3)]
        l0, l1, w1, b1, w2, b2, w3, b3 = self._keep
        s = _MLPStruct()
        s.ch = l0.shape[2]
        s.gw[0], s.gh[0] = l0.shape[1], l0.shape[0]
        s.gw[1], s.gh[1] = l1.shape[1], l1.shape[0]
        s.latent[0], s.latent[1] = l0.ctypes.data, l1.ctypes.data
        s.nin, s.hidden, s.nout = w1.shape[1], w1.shape[0], w3.shape[0]
        assert s.nin == 2 * s.ch and w2.shape == (s.hidden, s.hidden) and w3.shape[1] == s.hidden
        assert s.nin <= 64 and s.hidden <= 256 and s.nout <= 4
        s.w1, s.b1, s.w2, s.b2, s.w3, s.b3 = (a.ctypes.data for a in (w1, b1, w2, b2, w3, b3))
        s.saturate = 1 if saturate else 0
        self.struct = s
        self.latent_shapes = (l0.shape, l1.shape)

    @property
    def ref(self):
        return ctypes.byref(self.struct)


def mlp_features(mlp: MLP, Wt, Ht, x, y):
    f = np.zeros(mlp.struct.nin, np.float64)
    _load().oracle_mlp_features_f64(mlp.ref, Wt, Ht, x, y, _ptr(f))
    return f


def mlp_decode(mlp: MLP, Wt, Ht, xs, ys):
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    out = np.zeros((xs.size, 4), np.float64)
    _load().oracle_mlp_decode_f64(mlp.ref, Wt, Ht, xs.size, _ptr(xs), _ptr(ys), _ptr(out))
    return out


def mlp_loss_grad(mlp: MLP, Wt, Ht, xs, ys, targets):
    """Loss (1/B) sum (y - t)^2 and FP64 gradients of every parameter."""
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    t = np.ascontiguousarray(targets, dtype=np.float64)
    s = mlp.struct
    g = {"w1": np.zeros((s.hidden, s.nin)), "b1": np.zeros(s.hidden), "w2": np.zeros((s.hidden, s.hidden)),
         "b2": np.zeros(s.hidden), "w3": np.zeros((s.nout, s.hidden)), "b3": np.zeros(s.nout),
         "lat0": np.zeros(mlp.latent_shapes[0]), "lat1": np.zeros(mlp.latent_shapes[1])}
    loss = _load().oracle_mlp_loss_grad_f64(mlp.ref, Wt, Ht, xs.size, _ptr(xs), _ptr(ys), _ptr(t),
                                           *(_ptr(g[k]) for k in ("w1", "b1", "w2", "b2", "w3", "b3",
                                                                  "lat0", "lat1")))
    return loss, g


def filter_frame_learned_f64(mlp: MLP, Wt, Ht, uv, jac, coverage=None, *, view=0, alg=ALG_MASK, seed=0,
                             tile_w=8, tile_h=4, budget=32, mask_dim=16, edge_remap=1, group_tiles=0, fallback=0,
                             texels_per_lane=1, filter=0, y_offset=0):
    """Same selection as filter_frame, texel values from the FP64 MLP, filter in FP64."""
    uv = np.ascontiguousarray(uv, dtype=np.float32)
    jac = np.ascontiguousarray(jac, dtype=np.float32)
    H, W = uv.shape[0], uv.shape[1]
    cov = None if coverage is None else np.ascontiguousarray(coverage, dtype=np.uint8)
    out = np.zeros((H, W, 4), np.float64)
    ev = np.zeros((H, W), np.uint8)
    stats = np.zeros(9, np.int64)
    rc = _load().oracle_filter_learned_f64(mlp.ref, Wt, Ht, _ptr(uv), _ptr(jac), _ptr(cov), W, H, view, alg,
                                           seed, tile_w, tile_h, budget, mask_dim, edge_remap, group_tiles,
                                           fallback, texels_per_lane, filter, y_offset, _ptr(out),
                                           _ptr(ev), None, None, _ptr(stats))
    if rc != 0:
        raise ValueError(f"oracle_filter_learned_f64 rejected its arguments (rc={rc})")
    return out, ev, dict(zip(STAT_NAMES, (int(v) for v in stats)))
