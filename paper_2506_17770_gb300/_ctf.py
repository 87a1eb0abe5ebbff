"""Thin ctypes binding of the C ABI in include/ctf.h.

Argument marshalling only: every step of the filtering path runs in the CUDA
library (_build/libctf.so).  There is no CPU fallback: if the library is not
built, loading raises.  Tensors are torch tensors on the current CUDA device
(or host tensors for the *_host entry points); their data pointers are passed
through unchanged.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
RELEASE_LIB_PATH = os.path.join(_HERE, "_build", "libctf.so")
DEBUG_LIB_PATH = os.path.join(_HERE, "_build", "libctf_debug.so")
# CTF_LIBRARY=debug in the environment loads the debug build (index checks
# in every kernel, reported as CTF_ERR_BOUNDS) instead of the release one.
LIB_PATH = DEBUG_LIB_PATH if os.environ.get("CTF_LIBRARY", "") == "debug" else RELEASE_LIB_PATH

CTF_OK, CTF_ERR_ARG, CTF_ERR_ALIGN, CTF_ERR_UNSUPPORTED = 0, -1, -2, -3
CTF_ERR_OOM, CTF_ERR_CUDA, CTF_ERR_TIMEOUT, CTF_ERR_CORRUPT = -4, -5, -6, -7
CTF_ERR_BOUNDS = -8
CTF_ALG_4TAP, CTF_ALG_STF, CTF_ALG_LIST_MERGE, CTF_ALG_BOX, CTF_ALG_MASK = 0, 1, 2, 3, 4
CTF_EVAL_BLOCK, CTF_EVAL_MLP_FP16, CTF_EVAL_MLP_FP8 = 0, 1, 2
ALGORITHMS = {"4tap": 0, "stf": 1, "list_merge": 2, "box": 3, "mask": 4}


class CtfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class ctf_texture_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("mode", ctypes.c_int),
                ("blocks", ctypes.c_void_p)]


class ctf_filter_opts(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("budget", ctypes.c_int),
                ("mask_dim", ctypes.c_int), ("edge_remap", ctypes.c_int), ("group_dedup", ctypes.c_int),
                ("fallback", ctypes.c_int), ("texels_per_lane", ctypes.c_int), ("filter", ctypes.c_int)]


class ctf_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "tiles_total", "tiles_empty", "tiles_direct", "tiles_success", "tiles_fallback_budget",
        "tiles_fallback_minified", "pixels_active", "texel_evals", "texel_evals_unique")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                                  "(run paper_2506_17770_gb300.build.build(debug=...))")
            lib = ctypes.CDLL(LIB_PATH)
            P, I, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
            lib.ctf_version.restype = ctypes.c_char_p
            lib.ctf_status_string.restype = ctypes.c_char_p
            lib.ctf_status_string.argtypes = [I]
            lib.ctf_last_error.restype = ctypes.c_char_p
            lib.ctf_texture_create.argtypes = [P, P]
            lib.ctf_texture_destroy.argtypes = [P]
            sig = [P, P, P, P, I, I, I, I, U64, P, P, P, P, P]
            lib.ctf_filter.argtypes = sig
            lib.ctf_filter_host.argtypes = sig
            lib.ctf_filter_host_noalloc.argtypes = sig
            for fn in ("ctf_texture_create", "ctf_texture_destroy", "ctf_filter", "ctf_filter_host",
                       "ctf_filter_host_noalloc"):
                getattr(lib, fn).restype = I
            _bind_optional(lib)
            _lib = lib
    return _lib


class ctf_mlp_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("mode", ctypes.c_int),
                ("latent_w", ctypes.c_int * 2), ("latent_h", ctypes.c_int * 2),
                ("latent", ctypes.c_void_p * 2),
                ("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("w2", ctypes.c_void_p),
                ("b2", ctypes.c_void_p), ("w3", ctypes.c_void_p), ("b3", ctypes.c_void_p),
                ("act_absmax", ctypes.c_void_p * 3)]


class ctf_mlp_params(ctypes.Structure):
    _fields_ = [("latent", ctypes.c_void_p * 2), ("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p),
                ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p), ("w3", ctypes.c_void_p),
                ("b3", ctypes.c_void_p), ("weight_scale", ctypes.c_void_p * 3),
                ("act_scale", ctypes.c_void_p * 3)]


def _bind_optional(lib):
    """Signatures of the entry points of the learned decode and later modules."""
    P, I, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
    table = {
        "ctf_texture_create_mlp": ([P, P], I),
        "ctf_mlp_export": ([P, P], I),
        "ctf_mlp_decode": ([P, P, I, P, P], I),
        "ctf_sync_check": ([P], I),
        "ctf_trainer_create": ([P, P, P], I),
        "ctf_trainer_destroy": ([P], I),
        "ctf_trainer_step": ([P, ctypes.c_int64, P], I),
        "ctf_trainer_steps_done": ([P], ctypes.c_int64),
        "ctf_trainer_gradients": ([P, P, I, P, P, P], I),
        "ctf_trainer_get_params": ([P, P], I),
        "ctf_trainer_set_params": ([P, P], I),
        "ctf_trainer_export": ([P, I, P], I),
        "ctf_trainer_save": ([P, ctypes.c_char_p], I),
        "ctf_trainer_load": ([P, ctypes.c_char_p, P], I),
        "ctf_texture_compare": ([P, P, P, P, P], I),
        "ctf_mlp_train": ([P, P, I, P, P, P], I),
        "ctf_checkpoint_save": ([P, ctypes.c_char_p], I),
        "ctf_checkpoint_load": ([ctypes.c_char_p, P], I),
        "ctf_stream_status": ([P], I),
        "ctf_filter_batch": ([P, I, I, U64, P, P, P], I),
        "ctf_batch_graph_create": ([P, I, I, U64, P, P], I),
        "ctf_batch_graph_launch": ([P, P], I),
        "ctf_batch_graph_destroy": ([P], I),
        "ctf_batch_autotune": ([P, I, I, U64, P, P, P, P], I),
        "ctf_debug_device_allocations": ([], ctypes.c_int64),
        "ctf_debug_live_allocations": ([], ctypes.c_int64),
        "ctf_debug_fail_allocations": ([I, I], I),
        "ctf_debug_build": ([], I),
        "ctf_debug_selftest_bounds": ([I, P], I),
    }
    for name, (argtypes, restype) in table.items():
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.argtypes, f.restype = argtypes, restype


def _check(rc: int):
    if rc != CTF_OK:
        lib = load()
        raise CtfError(rc, f"{lib.ctf_status_string(rc).decode()}: {lib.ctf_last_error().decode()}")


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(f"cannot take a data pointer of {type(t)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _opts(opts):
    if opts is None or isinstance(opts, ctf_filter_opts):
        return opts
    d = {"tile_w": 8, "tile_h": 4, "budget": 32, "mask_dim": 16, "edge_remap": 1, "group_dedup": 0, "fallback": 0,
         "texels_per_lane": 1, "filter": 0}
    d.update(opts)
    return ctf_filter_opts(**d)


def _alg(alg):
    return ALGORITHMS[alg] if isinstance(alg, str) else int(alg)


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def ctf_version() -> str:
    return load().ctf_version().decode()


def ctf_status_string(status: int) -> str:
    return load().ctf_status_string(status).decode()


def ctf_last_error() -> str:
    return load().ctf_last_error().decode()


def ctf_texture_create(width: int, height: int, blocks, mode: int = CTF_EVAL_BLOCK) -> ctypes.c_void_p:
    """Block texture from a uint8 tensor/array of (width/4)*(height/4)*8 bytes."""
    lib = load()
    desc = ctf_texture_desc(width, height, mode, _ptr(blocks))
    out = ctypes.c_void_p()
    _check(lib.ctf_texture_create(ctypes.byref(desc), ctypes.byref(out)))
    return out


def ctf_texture_destroy(tex) -> None:
    _check(load().ctf_texture_destroy(tex))


def ctf_filter(tex, uv, jac, coverage, width, height, view_id, alg, seed, opts, out_rgba, out_evals,
               stats: bool = False, stream=None):
    """Filter one view on device buffers.  Returns the stats dict when stats=True."""
    st = ctf_stats() if stats else None
    rc = load().ctf_filter(tex, _ptr(uv), _ptr(jac), _ptr(coverage), int(width), int(height), int(view_id),
                           _alg(alg), int(seed) % 2**64, ctypes.byref(_opts(opts)) if opts is not None else None,
                           _ptr(out_rgba), _ptr(out_evals), ctypes.byref(st) if st is not None else None,
                           _stream(stream))
    _check(rc)
    return st.as_dict() if st is not None else None


def ctf_filter_host(tex, uv, jac, coverage, width, height, view_id, alg, seed, opts, out_rgba, out_evals,
                    stats: bool = False, stream=None):
    """ctf_filter on host buffers: page-locked buffers in
    place (the kernel reads the inputs and writes the image in host memory;
    the counts come back in one copy), others staged through library-owned
    device buffers; synchronous."""
    st = ctf_stats() if stats else None
    rc = load().ctf_filter_host(tex, _ptr(uv), _ptr(jac), _ptr(coverage), int(width), int(height),
                                int(view_id), _alg(alg), int(seed) % 2**64,
                                ctypes.byref(_opts(opts)) if opts is not None else None, _ptr(out_rgba),
                                _ptr(out_evals), ctypes.byref(st) if st is not None else None, _stream(stream))
    _check(rc)
    return st.as_dict() if st is not None else None


def ctf_filter_host_noalloc(tex, uv, jac, coverage, width, height, view_id, alg, seed, opts, out_rgba, out_evals,
                            stats: bool = False, stream=None):
    """ctf_filter_host without device allocation: scratch in the library's
    fixed static device array (views up to about 798,000 pixels)."""
    st = ctf_stats() if stats else None
    rc = load().ctf_filter_host_noalloc(tex, _ptr(uv), _ptr(jac), _ptr(coverage), int(width), int(height),
                                        int(view_id), _alg(alg), int(seed) % 2**64,
                                        ctypes.byref(_opts(opts)) if opts is not None else None, _ptr(out_rgba),
                                        _ptr(out_evals), ctypes.byref(st) if st is not None else None,
                                        _stream(stream))
    _check(rc)
    return st.as_dict() if st is not None else None


# ---------------------------------------------------------------------------
# Learned decode
# ---------------------------------------------------------------------------
def ctf_texture_create_mlp(width, height, mode, latents, w1, b1, w2, b2, w3, b3, act_absmax=None):
    """Learned-decode texture from FP32 parameters (numpy arrays or device
    tensors).  latents = (L0 [h0,w0,8], L1 [h1,w1,8])."""
    import numpy as np
    keep = []

    def arr(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            keep.append(a)
            return a.data_ptr()
        a = np.ascontiguousarray(a, dtype=np.float32)
        keep.append(a)
        return a.ctypes.data

    d = ctf_mlp_desc()
    d.width, d.height, d.mode = int(width), int(height), int(mode)
    for g in range(2):
        d.latent_h[g], d.latent_w[g] = int(latents[g].shape[0]), int(latents[g].shape[1])
        d.latent[g] = arr(latents[g])
    d.w1, d.b1, d.w2, d.b2, d.w3, d.b3 = (arr(a) for a in (w1, b1, w2, b2, w3, b3))
    if act_absmax is not None:
        for l in range(3):
            d.act_absmax[l] = arr(act_absmax[l])
    out = ctypes.c_void_p()
    _check(load().ctf_texture_create_mlp(ctypes.byref(d), ctypes.byref(out)))
    return out


def ctf_mlp_export(tex, latent_shapes, hidden=64, nin=16, nout=4):
    """The stored (quantised) parameters as float32 numpy arrays."""
    import numpy as np
    res = {"lat0": np.zeros(latent_shapes[0], np.float32), "lat1": np.zeros(latent_shapes[1], np.float32),
           "w1": np.zeros((hidden, nin), np.float32), "b1": np.zeros(hidden, np.float32),
           "w2": np.zeros((hidden, hidden), np.float32), "b2": np.zeros(hidden, np.float32),
           "w3": np.zeros((nout, hidden), np.float32), "b3": np.zeros(nout, np.float32),
           "ws0": np.zeros(hidden, np.float32), "ws1": np.zeros(hidden, np.float32),
           "ws2": np.zeros(nout, np.float32), "as0": np.zeros(nin, np.float32),
           "as1": np.zeros(hidden, np.float32), "as2": np.zeros(hidden, np.float32)}
    p = ctf_mlp_params()
    p.latent[0], p.latent[1] = res["lat0"].ctypes.data, res["lat1"].ctypes.data
    p.w1, p.b1, p.w2, p.b2, p.w3, p.b3 = (res[k].ctypes.data for k in ("w1", "b1", "w2", "b2", "w3", "b3"))
    for l in range(3):
        p.weight_scale[l] = res[f"ws{l}"].ctypes.data
        p.act_scale[l] = res[f"as{l}"].ctypes.data
    _check(load().ctf_mlp_export(tex, ctypes.byref(p)))
    return res


def ctf_mlp_decode(tex, xy, n, out_rgba, stream=None):
    _check(load().ctf_mlp_decode(tex, _ptr(xy), int(n), _ptr(out_rgba), _stream(stream)))


def ctf_sync_check(stream=None):
    _check(load().ctf_sync_check(_stream(stream)))


def ctf_stream_status(stream=None):
    """ctf_sync_check under the interface's other name."""
    _check(load().ctf_stream_status(_stream(stream)))


def ctf_selftest_bounded_wait(polls, stream=None):
    """Launch the bounded-wait self-test (a wait that runs out after `polls`
    tries and records CTF_ERR_TIMEOUT for the next ctf_sync_check)."""
    _check(load().ctf_selftest_bounded_wait(ctypes.c_uint32(int(polls)), _stream(stream)))


def ctf_debug_device_allocations():
    """Device allocations the library has attempted in this process."""
    return int(load().ctf_debug_device_allocations())


def ctf_debug_live_allocations():
    """Device allocations of the library that are currently held."""
    return int(load().ctf_debug_live_allocations())


def ctf_debug_fail_allocations(n, skip=0):
    """Let the library's next `skip` device allocations through, then make
    the n after them fail (CTF_ERR_OOM); n = 0 disarms."""
    _check(load().ctf_debug_fail_allocations(int(skip), int(n)))


def ctf_debug_build() -> bool:
    """True when the loaded library is the debug build (index checks)."""
    return bool(load().ctf_debug_build())


def ctf_debug_selftest_bounds(index, stream=None):
    """One thread reads element `index` of a 32-int shared array through the
    debug build's index check; an index outside [0, 32) is recorded and the
    next ctf_sync_check raises CTF_ERR_BOUNDS.  The release library refuses
    (CTF_ERR_UNSUPPORTED)."""
    _check(load().ctf_debug_selftest_bounds(int(index), _stream(stream)))


# ---------------------------------------------------------------------------
# Training
# ---------------------------------------------------------------------------
class ctf_train_desc(ctypes.Structure):
    _fields_ = [("latent_w", ctypes.c_int * 2), ("latent_h", ctypes.c_int * 2), ("batch", ctypes.c_int),
                ("total_steps", ctypes.c_int64), ("lr_weights", ctypes.c_float), ("lr_latents", ctypes.c_float),
                ("lr_final_frac", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("seed", ctypes.c_uint64)]


class ctf_mlp_arrays(ctypes.Structure):
    _fields_ = [("latent", ctypes.c_void_p * 2), ("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p),
                ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p), ("w3", ctypes.c_void_p),
                ("b3", ctypes.c_void_p)]


PARAM_NAMES = ("lat0", "lat1", "w1", "b1", "w2", "b2", "w3", "b3")


def train_desc(latent_sizes, batch, total_steps, lr_weights=3e-3, lr_latents=3e-2, lr_final_frac=0.1,
               beta1=0.9, beta2=0.99, eps=1e-10, seed=3):
    """latent_sizes = ((w0, h0), (w1, h1))."""
    d = ctf_train_desc()
    for g in range(2):
        d.latent_w[g], d.latent_h[g] = int(latent_sizes[g][0]), int(latent_sizes[g][1])
    d.batch, d.total_steps = int(batch), int(total_steps)
    d.lr_weights, d.lr_latents, d.lr_final_frac = lr_weights, lr_latents, lr_final_frac
    d.beta1, d.beta2, d.eps, d.seed = beta1, beta2, eps, int(seed) % 2**64
    return d


def _param_arrays(desc, dtype="float32"):
    import numpy as np
    shapes = {"lat0": (desc.latent_h[0], desc.latent_w[0], 8), "lat1": (desc.latent_h[1], desc.latent_w[1], 8),
              "w1": (64, 16), "b1": (64,), "w2": (64, 64), "b2": (64,), "w3": (4, 64), "b3": (4,)}
    return {k: np.zeros(v, dtype) for k, v in shapes.items()}


def _arrays_struct(d):
    a = ctf_mlp_arrays()
    a.latent[0], a.latent[1] = d["lat0"].ctypes.data, d["lat1"].ctypes.data
    a.w1, a.b1, a.w2, a.b2, a.w3, a.b3 = (d[k].ctypes.data for k in ("w1", "b1", "w2", "b2", "w3", "b3"))
    return a


def ctf_trainer_create(exact_tex, desc):
    out = ctypes.c_void_p()
    _check(load().ctf_trainer_create(exact_tex, ctypes.byref(desc), ctypes.byref(out)))
    return out


def ctf_trainer_destroy(tr):
    _check(load().ctf_trainer_destroy(tr))


def ctf_trainer_step(tr, steps, stream=None):
    _check(load().ctf_trainer_step(tr, int(steps), _stream(stream)))


def ctf_trainer_steps_done(tr):
    return int(load().ctf_trainer_steps_done(tr))


def ctf_trainer_gradients(tr, desc, xy, n, stream=None):
    """(loss, dict of float32 gradient arrays) for device int32 texels xy [n,2]."""
    g = _param_arrays(desc)
    loss = ctypes.c_double()
    a = _arrays_struct(g)
    _check(load().ctf_trainer_gradients(tr, _ptr(xy), int(n), ctypes.byref(loss), ctypes.byref(a),
                                        _stream(stream)))
    return loss.value, g


def ctf_trainer_get_params(tr, desc):
    p = _param_arrays(desc)
    a = _arrays_struct(p)
    _check(load().ctf_trainer_get_params(tr, ctypes.byref(a)))
    return p


def ctf_trainer_set_params(tr, params):
    import numpy as np
    p = {k: np.ascontiguousarray(v, dtype=np.float32) for k, v in params.items()}
    a = _arrays_struct(p)
    _check(load().ctf_trainer_set_params(tr, ctypes.byref(a)))


def ctf_trainer_export(tr, mode):
    out = ctypes.c_void_p()
    _check(load().ctf_trainer_export(tr, int(mode), ctypes.byref(out)))
    return out


def ctf_trainer_save(tr, path):
    _check(load().ctf_trainer_save(tr, path.encode()))


def ctf_trainer_load(exact_tex, path):
    out = ctypes.c_void_p()
    _check(load().ctf_trainer_load(exact_tex, path.encode(), ctypes.byref(out)))
    return out


def ctf_texture_compare(exact_tex, learned_tex, stream=None):
    """(mse over RGB, max abs channel error) of a learned texture vs the exact one."""
    mse, mx = ctypes.c_double(), ctypes.c_double()
    _check(load().ctf_texture_compare(exact_tex, learned_tex, ctypes.byref(mse), ctypes.byref(mx),
                                      _stream(stream)))
    return mse.value, mx.value


class ctf_train_report(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("texels", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("mse_rgb", ctypes.c_double), ("max_abs", ctypes.c_double), ("psnr_db", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def ctf_mlp_train(exact_tex, desc, mode, stream=None):
    """Train, export and compare in one call: (learned texture, report dict)."""
    out = ctypes.c_void_p()
    rep = ctf_train_report()
    _check(load().ctf_mlp_train(exact_tex, ctypes.byref(desc), int(mode), ctypes.byref(out), ctypes.byref(rep),
                                _stream(stream)))
    return out, rep.as_dict()


def ctf_checkpoint_save(tex, path):
    _check(load().ctf_checkpoint_save(tex, path.encode()))


def ctf_checkpoint_load(path):
    out = ctypes.c_void_p()
    _check(load().ctf_checkpoint_load(path.encode(), ctypes.byref(out)))
    return out


# ---------------------------------------------------------------------------
# Batched views
# ---------------------------------------------------------------------------
class ctf_view(ctypes.Structure):
    _fields_ = [("tex", ctypes.c_void_p), ("uv", ctypes.c_void_p), ("jac", ctypes.c_void_p),
                ("coverage", ctypes.c_void_p), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("view_id", ctypes.c_int), ("out_rgba", ctypes.c_void_p), ("out_evals", ctypes.c_void_p)]


class ctf_batch_opts(ctypes.Structure):
    _fields_ = [("filter", ctf_filter_opts), ("items_per_fetch", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("solo_tiles", ctypes.c_int)]

    def as_dict(self):
        f = self.filter
        return {"tile_w": f.tile_w, "tile_h": f.tile_h, "budget": f.budget, "mask_dim": f.mask_dim,
                "edge_remap": f.edge_remap, "group_dedup": f.group_dedup, "fallback": f.fallback,
                "texels_per_lane": f.texels_per_lane,
                "items_per_fetch": self.items_per_fetch,
                "ctas_per_sm": self.ctas_per_sm, "solo_tiles": self.solo_tiles}


def batch_opts(tile_w=8, tile_h=4, budget=32, mask_dim=16, edge_remap=1, items_per_fetch=4, ctas_per_sm=4,
               group_dedup=0, fallback=0, texels_per_lane=1, solo_tiles=16384):
    o = ctf_batch_opts()
    o.filter = ctf_filter_opts(tile_w, tile_h, budget, mask_dim, edge_remap, group_dedup, fallback, texels_per_lane)
    o.items_per_fetch, o.ctas_per_sm, o.solo_tiles = items_per_fetch, ctas_per_sm, solo_tiles
    return o


def views_array(views):
    """views: list of dicts with tex, uv, jac, coverage, width, height, view_id, out_rgba, out_evals."""
    arr = (ctf_view * len(views))()
    for i, v in enumerate(views):
        arr[i] = ctf_view(v["tex"].value if hasattr(v["tex"], "value") else v["tex"], _ptr(v["uv"]), _ptr(v["jac"]),
                          _ptr(v.get("coverage")), int(v["width"]), int(v["height"]), int(v.get("view_id", i)),
                          _ptr(v["out_rgba"]), _ptr(v.get("out_evals")))
    return arr


def ctf_filter_batch(views, alg, seed, opts=None, stats=False, stream=None):
    arr = views if isinstance(views, ctypes.Array) else views_array(views)
    st = ctf_stats() if stats else None
    _check(load().ctf_filter_batch(arr, len(arr), _alg(alg), int(seed) % 2**64,
                                   ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(st) if st is not None else None, _stream(stream)))
    return st.as_dict() if st is not None else None


def ctf_batch_graph_create(views, alg, seed, opts=None):
    arr = views if isinstance(views, ctypes.Array) else views_array(views)
    out = ctypes.c_void_p()
    _check(load().ctf_batch_graph_create(arr, len(arr), _alg(alg), int(seed) % 2**64,
                                         ctypes.byref(opts) if opts is not None else None, ctypes.byref(out)))
    return out


def ctf_batch_graph_launch(g, stream=None):
    _check(load().ctf_batch_graph_launch(g, _stream(stream)))


def ctf_batch_graph_destroy(g):
    _check(load().ctf_batch_graph_destroy(g))


def ctf_batch_autotune(views, alg, seed, base=None, stream=None):
    arr = views if isinstance(views, ctypes.Array) else views_array(views)
    best = ctf_batch_opts()
    ms = ctypes.c_double()
    _check(load().ctf_batch_autotune(arr, len(arr), _alg(alg), int(seed) % 2**64,
                                     ctypes.byref(base) if base is not None else None, ctypes.byref(best),
                                     ctypes.byref(ms), _stream(stream)))
    return best, ms.value
