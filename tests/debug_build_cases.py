"""Parity cases for the debug build of the CUDA library.

`run_cases()` runs a fixed, seeded set of calls through the C ABI and
returns every output array by case name: the exact decode on the 128x128
magnified plane and on ragged frames (every algorithm, the option sets of the
parity tests, fallbacks C / C+, two texels per lane, the bicubic filters,
rotated quads whose tiles hold up to 54 texels), the learned decode in FP16
and FP8 (every kernel: per-pixel 4-tap, List Merge, the packed groups with
and without group_dedup, the extension kernel), the batch of block and
learned views, the texel decode, and gradients and steps of the trainer.
After every call the device error word is read (ctf_sync_check), so an index
check of the debug build that fired fails the call it fired in.  The exact
decode's outputs are also compared with the oracle here.

Run as a script with CTF_LIBRARY=debug (the debug library), it writes the
outputs to the .npz named by its argument; tests/test_gpu_debug_build.py
compares them bit for bit with the release library's.  With the argument
`selftest` it exercises ctf_debug_selftest_bounds instead."""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2506_17770_gb300 import _ctf, synth  # noqa: E402

ALGS = {"4tap": 0, "stf": 1, "list_merge": 2, "box": 3, "mask": 4}
COLLAB = ("list_merge", "box", "mask")


def _torch():
    import torch
    return torch


def _mixed_scene(W, H, seed, Wt=64):
    """Tiles of random rotation and magnification in [0.6, 8], some over the
    texture's edge, 20% of the pixels uncovered, a NaN, a huge coordinate
    and an infinite Jacobian entry."""
    g = np.random.default_rng(seed)
    uv = np.zeros((H, W, 2))
    jac = np.zeros((H, W, 4))
    for ty in range(0, H, 4):
        for tx in range(0, W, 8):
            m = math.exp(g.uniform(math.log(0.6), math.log(8.0)))
            r = g.uniform(0, 2 * math.pi)
            c, s = math.cos(r), math.sin(r)
            o = g.uniform(-3, 60, 2)
            ly, lx = np.meshgrid(np.arange(4) + 0.5, np.arange(8) + 0.5, indexing="ij")
            X = (c * lx - s * ly) / m + o[0]
            Y = (s * lx + c * ly) / m + o[1]
            hh, ww = min(4, H - ty), min(8, W - tx)
            sl = (slice(ty, ty + hh), slice(tx, tx + ww))
            uv[sl + (0,)] = (X / Wt)[:hh, :ww]
            uv[sl + (1,)] = (Y / Wt)[:hh, :ww]
            jac[sl] = np.array([c / m / Wt, s / m / Wt, -s / m / Wt, c / m / Wt])
    cov = (g.uniform(size=(H, W)) > 0.2).astype(np.uint8)
    uv = uv.astype(np.float32)
    jac = jac.astype(np.float32)
    if H > 1 and W > 1:
        uv[0, 0] = np.nan
        uv[H // 2, W // 3] = [3e7, 0.5]
        jac[H - 1, W - 1] = np.inf
    return uv, jac, cov


def _quads():
    q = synth.rotated_quad_tiles(1.001, np.arange(0, 91, 3.0), 8, Wt=64, Ht=64)
    uv = (q.uv.astype(np.float64) - 996.0 / 64.0).astype(np.float32)
    return uv, q.jac.astype(np.float32)


def _filter(tex, uv, jac, cov, alg, opts, seed):
    torch = _torch()
    H, W = uv.shape[:2]
    d_uv = torch.from_numpy(np.ascontiguousarray(uv)).cuda()
    d_jac = torch.from_numpy(np.ascontiguousarray(jac)).cuda()
    d_cov = None if cov is None else torch.from_numpy(np.ascontiguousarray(cov)).cuda()
    out = torch.full((H, W, 4), -7.0, dtype=torch.float32, device="cuda")
    ev = torch.full((H, W), 99, dtype=torch.uint8, device="cuda")
    st = _ctf.ctf_filter(tex, d_uv, d_jac, d_cov, W, H, 0, alg, seed, opts, out, ev, stats=True)
    _ctf.ctf_sync_check()
    stats = np.array([st[k] for k in sorted(st)], np.int64)
    return out.cpu().numpy(), ev.cpu().numpy(), stats


def _oracle_opts(opts):
    o = {"tile_w": 8, "tile_h": 4, "budget": 32, "mask_dim": 16, "edge_remap": 1}
    for k, v in (opts or {}).items():
        o[k] = v
    return o


def _check_exact(blocks, Wt, Ht, uv, jac, cov, alg, opts, seed, got):
    o = _oracle_opts(opts)
    ref, ref_ev, ref_st = oracle.filter_frame(blocks, Wt, Ht, uv, jac, cov, alg=ALGS[alg], seed=seed, **o)[:3]
    out, ev, st = got
    if not (np.array_equal(ev, ref_ev) and np.array_equal(out.view(np.uint32), ref.view(np.uint32))
            and np.array_equal(st, np.array([ref_st[k] for k in sorted(ref_st)], np.int64))):
        raise AssertionError(f"exact decode differs from the oracle: {alg} {opts}")


EXACT_OPTS = [None, {"edge_remap": 0}, {"budget": 9, "mask_dim": 11}, {"tile_w": 16, "tile_h": 2, "budget": 20},
              {"tile_w": 4, "tile_h": 8}]
EXT_OPTS = [{"fallback": 1}, {"fallback": 2, "mask_dim": 11}, {"texels_per_lane": 2, "budget": 64},
            {"texels_per_lane": 2, "budget": 40, "fallback": 2, "tile_w": 16, "tile_h": 2}]
BICUBIC_OPTS = [{"filter": 1}, {"filter": 2, "mask_dim": 11, "tile_w": 4, "tile_h": 8}]
LEARNED_OPTS = [None, {"tile_w": 4, "tile_h": 8, "mask_dim": 11}, {"group_dedup": 1}, {"fallback": 1},
                {"fallback": 2}, {"texels_per_lane": 2, "budget": 64},
                {"texels_per_lane": 2, "budget": 64, "fallback": 2, "mask_dim": 11}]


def _learned_params(seed, Wt, Ht):
    g = np.random.default_rng(seed)
    lat = [g.normal(0, 1.0, (Ht // 4, Wt // 4, 8)).astype(np.float32),
           g.normal(0, 1.0, (Ht // 8, Wt // 8, 8)).astype(np.float32)]
    p = (g.normal(0, math.sqrt(2 / 16), (64, 16)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
         g.normal(0, math.sqrt(2 / 64), (64, 64)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
         g.normal(0, 0.04, (4, 64)).astype(np.float32), np.array([0.5, 0.45, 0.55, 0.9], np.float32))
    return lat, p


def _act_absmax(lat, p, Wt, Ht):
    """Per-channel ranges of the FP64 network's layer inputs over every
    texel, times 1.1 (the E4M3 activation scales)."""
    full = oracle.MLP((lat[0], lat[1]), *p)
    F = np.stack([oracle.mlp_features(full, Wt, Ht, x, y) for y in range(Ht) for x in range(Wt)])
    h1 = np.maximum(F @ p[0].T.astype(np.float64) + p[1], 0)
    h2 = np.maximum(h1 @ p[2].T.astype(np.float64) + p[3], 0)
    return [(1.1 * np.abs(a).max(axis=0) + 1e-3).astype(np.float32) for a in (F, h1, h2)]


def run_cases() -> dict:
    torch = _torch()
    oracle.build()
    res = {}

    def put(name, got):
        res[name + ":rgba"], res[name + ":evals"], res[name + ":stats"] = got

    # ---- exact decode
    blocks = synth.random_blocks(64, 64, seed=7)
    tex = _ctf.ctf_texture_create(64, 64, blocks)
    try:
        plane = synth.magnified_plane(128, 128, 64, 64, scale=0.25)
        for alg in ALGS:
            for tw, th in ((8, 4), (4, 8), (16, 2)):
                opts = {"tile_w": tw, "tile_h": th}
                got = _filter(tex, plane.uv, plane.jac, None, alg, opts, 0)
                _check_exact(blocks, 64, 64, plane.uv, plane.jac, None, alg, opts, 0, got)
                put(f"exact128:{alg}:{tw}x{th}", got)
        for W, H in ((133, 77), (17, 3), (250, 131), (1, 1), (8, 4)):
            uv, jac, cov = _mixed_scene(W, H, W * 1000 + H)
            for alg in ALGS:
                opt_sets = EXACT_OPTS + BICUBIC_OPTS + (EXT_OPTS if alg in COLLAB else [])
                for i, opts in enumerate(opt_sets):
                    got = _filter(tex, uv, jac, cov, alg, opts, 77)
                    _check_exact(blocks, 64, 64, uv, jac, cov, alg, opts, 77, got)
                    put(f"exact{W}x{H}:{alg}:{i}", got)
        quv, qjac = _quads()
        for alg in COLLAB:
            opts = {"texels_per_lane": 2, "budget": 64}
            got = _filter(tex, quv, qjac, None, alg, opts, 0)
            _check_exact(blocks, 64, 64, quv, qjac, None, alg, opts, 0, got)
            put(f"exactquads:{alg}", got)
    finally:
        _ctf.ctf_texture_destroy(tex)

    # ---- learned decode, FP16 and FP8
    lat, p = _learned_params(1, 64, 64)
    for mode, tag in ((_ctf.CTF_EVAL_MLP_FP16, "fp16"), (_ctf.CTF_EVAL_MLP_FP8, "fp8")):
        amax = _act_absmax(lat, p, 64, 64) if mode == _ctf.CTF_EVAL_MLP_FP8 else None
        ltex = _ctf.ctf_texture_create_mlp(64, 64, mode, lat, *p, act_absmax=amax)
        try:
            plane = synth.magnified_plane(128, 128, 64, 64, scale=0.25)
            for alg in ALGS:
                put(f"{tag}128:{alg}", _filter(ltex, plane.uv, plane.jac, None, alg, None, 0))
            uv, jac, cov = _mixed_scene(133, 70, 23)
            for alg in ALGS:
                for i, opts in enumerate(LEARNED_OPTS):
                    if alg not in COLLAB and i >= 3 or alg == "4tap" and i == 2:
                        continue
                    put(f"{tag}133x70:{alg}:{i}", _filter(ltex, uv, jac, cov, alg, opts, 5))
            quv, qjac = _quads()
            for md in (16, 11):
                put(f"{tag}quads:{md}", _filter(ltex, quv, qjac, None, "mask",
                                                {"texels_per_lane": 2, "budget": 64, "mask_dim": md}, 0))
            xy = torch.stack(torch.meshgrid(torch.arange(64), torch.arange(64), indexing="xy"), -1)
            xy = xy.reshape(-1, 2).to(torch.int32).cuda().contiguous()
            dec = torch.empty((64 * 64, 4), dtype=torch.float32, device="cuda")
            _ctf.ctf_mlp_decode(ltex, xy, 64 * 64, dec)
            _ctf.ctf_sync_check()
            res[f"{tag}decode"] = dec.cpu().numpy()
        finally:
            _ctf.ctf_texture_destroy(ltex)

    # ---- batch of block and learned views (persistent kernels and solo views)
    btex = _ctf.ctf_texture_create(64, 64, blocks)
    ltex = _ctf.ctf_texture_create_mlp(64, 64, _ctf.CTF_EVAL_MLP_FP16, lat, *p)
    try:
        views, keep = [], []
        for i, (W, H) in enumerate(((133, 77), (17, 3), (250, 131), (64, 64), (96, 40), (40, 96))):
            uv, jac, cov = _mixed_scene(W, H, 500 + i)
            d = {"uv": torch.from_numpy(uv).cuda(), "jac": torch.from_numpy(jac).cuda(),
                 "coverage": torch.from_numpy(cov).cuda(),
                 "out_rgba": torch.full((H, W, 4), -7.0, device="cuda"),
                 "out_evals": torch.full((H, W), 99, dtype=torch.uint8, device="cuda")}
            keep.append(d)
            views.append(dict(d, tex=btex if i % 2 == 0 else ltex, width=W, height=H, view_id=i))
        for alg in ("mask", "box", "list_merge", "4tap"):
            for solo in (16384, 8):
                st = _ctf.ctf_filter_batch(views, alg, 11, _ctf.batch_opts(solo_tiles=solo), stats=True)
                _ctf.ctf_sync_check()
                for i, d in enumerate(keep):
                    res[f"batch:{alg}:{solo}:{i}:rgba"] = d["out_rgba"].cpu().numpy()
                    res[f"batch:{alg}:{solo}:{i}:evals"] = d["out_evals"].cpu().numpy()
                res[f"batch:{alg}:{solo}:stats"] = np.array([st[k] for k in sorted(st)], np.int64)
    finally:
        _ctf.ctf_texture_destroy(btex)
        _ctf.ctf_texture_destroy(ltex)

    # ---- trainer: gradients on explicit texels, then Philox-sampled steps
    ttex = _ctf.ctf_texture_create(64, 64, blocks)
    try:
        desc = _ctf.train_desc(((16, 16), (8, 8)), batch=1000, total_steps=8)
        tr = _ctf.ctf_trainer_create(ttex, desc)
        try:
            g = np.random.default_rng(3)
            xy = torch.from_numpy(g.integers(-2, 66, (700, 2)).astype(np.int32)).cuda()
            loss, grads = _ctf.ctf_trainer_gradients(tr, desc, xy, 700)
            _ctf.ctf_sync_check()
            res["train:loss"] = np.array([loss])
            for k, v in grads.items():
                res[f"train:grad:{k}"] = v
            _ctf.ctf_trainer_step(tr, 4)
            _ctf.ctf_sync_check()
            for k, v in _ctf.ctf_trainer_get_params(tr, desc).items():
                res[f"train:param:{k}"] = v
        finally:
            _ctf.ctf_trainer_destroy(tr)
    finally:
        _ctf.ctf_texture_destroy(ttex)
    return res


def selftest() -> dict:
    """ctf_debug_selftest_bounds on indices inside and outside [0, 32)."""
    out = {"debug_build": _ctf.ctf_debug_build()}
    for index in (0, 31, 32, 40, -1, 7):
        _ctf.ctf_debug_selftest_bounds(index)
        try:
            _ctf.ctf_sync_check()
            out[str(index)] = {"status": 0, "message": ""}
        except _ctf.CtfError as e:
            out[str(index)] = {"status": e.status, "message": str(e)}
    return out


if __name__ == "__main__":
    if sys.argv[1] == "selftest":
        print(json.dumps(selftest()))
    else:
        if not _ctf.ctf_debug_build():
            raise SystemExit("CTF_LIBRARY=debug is not set: the release library was loaded")
        r = run_cases()
        np.savez(sys.argv[1], **r)
        print(json.dumps({"cases": len(r)}))
