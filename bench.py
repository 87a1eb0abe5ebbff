#!/usr/bin/env python3
"""Throughput of collaborative texture filtering on one GB300 (or N, one
process per GPU, each filtering its own view: weak scaling, no collective on
the data path).

Workload (default "frame1080"): one 1920x1080 view of a perspective ground
plane plus three tilted quads (magnification about 0.1 to 20, 9.5% of pixels
minified), texture 2048x2048 in 4x4-texel blocks with seeded random endpoints
and indices.  A step filters the whole view with the headline collaborative
algorithm (Mask Sampling, 11x11 mask, one-tap STF fallback, 8x4 warps).  The
same view is also timed with per-pixel 4-tap bilinear, Box Sampling, List
Merge and the 16x16 mask, each reported beside the headline.

Timing: W warm-up steps, then K timed steps; before every step a 256 MiB
buffer is written to flush L2 (the view's I/O, 87 MB, would otherwise stay in
the 129 MB L2) and a second 256 MiB buffer is read, so that L2 holds clean
lines and the timed kernel does not pay for writing back the flush's dirty
ones; each step's kernel is timed with CUDA events on the launching stream.
One JSON line on rank 0.

--impl reference times the CPU oracle (plain C, one thread) on the same view
and algorithm: each step is one full view.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filtered pixels/s and texel evals/pixel, collaborative vs 4-tap on one GB300 at tol"
HEADLINE = ("mask", {"tile_w": 8, "tile_h": 4, "budget": 32, "mask_dim": 11, "edge_remap": 1})
OTHERS = [("4tap", "4tap", {}), ("box", "box", {}), ("list_merge", "list_merge", {}),
          ("mask16", "mask", {"mask_dim": 16}),
          ("mask11_fallback_c", "mask", {"fallback": 1}), ("mask11_fallback_cplus", "mask", {"fallback": 2}),
          ("mask11_two_texels_per_lane", "mask", {"texels_per_lane": 2, "budget": 64}),
          ("bspline_16tap", "4tap", {"filter": 1}), ("bspline_mask16", "mask", {"filter": 1, "mask_dim": 16}),
          ("catmull_rom_16tap", "4tap", {"filter": 2}), ("catmull_rom_mask16", "mask", {"filter": 2, "mask_dim": 16})]
ALG_ID = {"4tap": 0, "stf": 1, "list_merge": 2, "box": 3, "mask": 4}
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["frame1080", "frame2160", "plane128"], default="frame1080")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline only (for profiling)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-decode workload")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-views workload")
    ap.add_argument("--train-steps", type=int, default=8192, help="training steps (learned)")
    ap.add_argument("--train-batch", type=int, default=8192, help="texels per training step (learned)")
    return ap.parse_args()


def workload(name: str, rank: int):
    from paper_2506_17770_gb300 import synth
    seed = synth.SEED_SCENE + rank
    if name == "plane128":
        Wt = Ht = 64
        sc = synth.magnified_plane(128, 128, Wt, Ht, scale=0.25, seed=seed)
        desc = "128x128 magnified plane (4x), texture 64x64 random blocks"
    elif name == "frame2160":
        Wt = Ht = 2048
        sc = synth.ground_plane_with_quads(3840, 2160, Wt, Ht, seed=seed)
        desc = "3840x2160 ground plane + 3 tilted quads, texture 2048x2048 random blocks"
    else:
        Wt = Ht = 2048
        sc = synth.ground_plane_with_quads(1920, 1080, Wt, Ht, seed=seed)
        desc = "1920x1080 ground plane + 3 tilted quads, texture 2048x2048 random blocks"
    blocks = synth.random_blocks(Wt, Ht, seed=synth.SEED_TEXTURE)
    return sc, blocks, Wt, Ht, desc


def algorithmic_bytes(alg: str, npix: int, tex_bytes: int, has_cov: bool) -> int:
    """Bytes a kernel must move: per pixel uv 8 + (jac 16 for the collaborative
    algorithms, which vote on minification) + coverage 1 + RGBA32F 16 + count 1,
    plus the texture read once."""
    per = 8 + 16 + 1 + (1 if has_cov else 0)
    if alg not in ("4tap", "stf"):
        per += 16
    return npix * per + tex_bytes


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def measured_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured burst bf16"
    except Exception:
        return 1900.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("ctf_filter.cu", "ctf_device.cuh", "ctf_exact_tile.cuh", "ctf_select.cuh"):
        with open(os.path.join(ROOT, "paper_2506_17770_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload_name: str, alg_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(f"{workload_name}:{alg_key}")
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return int(e["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_cpu_oracle(sc, blocks, Wt, Ht, alg, opts, seconds: float, max_frames: int = 1000):
    import oracle
    o = {"tile_w": 8, "tile_h": 4, "budget": 32, "mask_dim": 16, "edge_remap": 1}
    o.update(opts)
    frames, t0 = 0, time.perf_counter()
    ev_total = 0
    while True:
        _, ev, st = oracle.filter_frame(blocks, Wt, Ht, sc.uv, sc.jac, sc.coverage, view=0, alg=ALG_ID[alg],
                                        seed=0, **o)
        frames += 1
        ev_total += st["texel_evals"]
        el = time.perf_counter() - t0
        if el >= seconds or frames >= max_frames:
            break
    return frames, el, ev_total


def _psnr(img, ref):
    """PSNR of RGB in [0, 1] (alpha excluded), log10."""
    import torch
    mse = torch.mean((img[..., :3] - ref[..., :3]) ** 2).item()
    return -10 * math.log10(max(mse, 1e-30))


class L2Flush:
    """Writes a 256 MiB buffer (evicting everything from the 129 MB L2), then
    reads another 256 MiB so that the lines left in L2 are clean."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        self.r = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def __call__(self):
        self.w.zero_()
        self.r.sum()


def _timed_views(launch, steps, warmup, flush, stream):
    """Sum of per-launch CUDA-event times (ms) with L2 flushed before each."""
    import torch
    for _ in range(warmup):
        if flush is not None:
            flush()
        launch()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        if flush is not None:
            flush()
        a.record(stream)
        launch()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev)


def bench_learned(args, dev, stream, flush, peaks):
    """Learned texel decode: a 4096^2 procedural texture (6 octaves of
    gradient noise + checker edges), block-encoded, learned by the library's
    trainer into two latent grids (1024^2, 512^2, 8 ch) and a 16-64-64-4 MLP
    from texels of its exact decode (`--train-steps` x `--train-batch`
    texels, 8192 x 8192 = 64M by default); then a 3840x2160 view
    with magnification log-uniform in [1, 16] filtered with the learned
    decode (FP16 and FP8) by per-pixel 4-tap and the collaborative
    algorithms."""
    import numpy as np
    import torch
    import oracle
    from paper_2506_17770_gb300 import _ctf, synth
    res = {}
    t0 = time.perf_counter()
    rgba = synth.procedural_rgba8(4096, device=dev)
    blocks = synth.encode_blocks(rgba)
    res["input_gen_s"] = time.perf_counter() - t0
    exact = _ctf.ctf_texture_create(4096, 4096, blocks)
    steps, batch = args.train_steps, args.train_batch
    desc = _ctf.train_desc(((1024, 1024), (512, 512)), batch=batch, total_steps=steps, lr_weights=1e-2,
                           lr_latents=1e-1, lr_final_frac=0.02, seed=3)
    tr = _ctf.ctf_trainer_create(exact, desc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _ctf.ctf_trainer_step(tr, steps, stream=stream)
    _ctf.ctf_sync_check(stream)
    train_s = time.perf_counter() - t0
    res["training"] = {"steps": steps, "batch": batch, "texels": steps * batch, "seconds": train_s,
                       "texels_per_s": steps * batch / train_s,
                       "schedule": "Adam, lr 1e-2 (weights) / 1e-1 (latents), linear decay to 2% over all steps"}
    texs = {"fp16": _ctf.ctf_trainer_export(tr, _ctf.CTF_EVAL_MLP_FP16),
            "fp8": _ctf.ctf_trainer_export(tr, _ctf.CTF_EVAL_MLP_FP8)}
    for k, t in texs.items():
        mse, mx = _ctf.ctf_texture_compare(exact, t, stream=stream)
        res[f"{k}_texels_vs_exact"] = {"psnr_db": -10 * math.log10(max(mse, 1e-30)), "max_abs": mx}
    sc = synth.perspective_view(3840, 2160, 4096, 4096, 1.0, 16.0, seed=2)
    W, H = sc.W, sc.H
    npix = W * H
    uv = torch.from_numpy(sc.uv).to(dev)
    jac = torch.from_numpy(sc.jac).to(dev)
    cov = torch.from_numpy(sc.coverage).to(dev)
    out = torch.empty((H, W, 4), device=dev)
    ev = torch.empty((H, W), dtype=torch.uint8, device=dev)
    ref_exact = torch.empty((H, W, 4), device=dev)
    opts11 = {"mask_dim": 11}
    _ctf.ctf_filter(exact, uv, jac, cov, W, H, 0, "4tap", 0, None, ref_exact, ev, stream=stream)
    k = max(3, min(args.steps, 20))
    runs = {}
    for tname in ("fp16", "fp8"):
        tex = texs[tname]
        for name in ("4tap", "stf", "mask", "mask_group_dedup", "box", "list_merge"):
            if tname == "fp8" and name in ("stf", "box", "list_merge"):
                continue
            alg = "mask" if name.startswith("mask") else name
            o = opts11 if name == "mask" else ({"mask_dim": 11, "group_dedup": 1} if name == "mask_group_dedup"
                                              else None)
            ms = _timed_views(lambda: _ctf.ctf_filter(tex, uv, jac, cov, W, H, 0, alg, 0, o, out, ev,
                                                     stream=stream), k, 2, flush, stream)
            st = _ctf.ctf_filter(tex, uv, jac, cov, W, H, 0, alg, 0, o, out, ev, stats=True, stream=stream)
            _ctf.ctf_sync_check(stream)
            mse = torch.mean((out[..., :3] - ref_exact[..., :3]) ** 2).item()
            t = ms / k * 1e-3
            flops = st["texel_evals_unique"] * 10752  # evaluations done
            peak = peaks["bf16"] * (2.0 if tname == "fp8" else 1.0)
            runs[f"{tname}_{name}"] = {
                "pixels_per_s": npix / t, "ms_per_view": t * 1e3, "us_per_mpixel": t * 1e6 / (npix / 1e6),
                "evals_per_pixel": st["texel_evals"] / max(1, st["pixels_active"]),
                "evaluations_done_per_pixel": st["texel_evals_unique"] / max(1, st["pixels_active"]),
                "texel_evals_per_s": st["texel_evals"] / t,
                "psnr_vs_exact_4tap_db": -10 * math.log10(max(mse, 1e-30)),
                "tensor": {"achieved_tflops": flops / t / 1e12, "peak_tflops": peak,
                           "frac": flops / t / 1e12 / peak,
                           "peak_kind": peaks["bf16_kind"] + (" x2 (nominal fp8/bf16 ratio)" if tname == "fp8" else "")},
                "tiles_success": st["tiles_success"], "tiles_fallback_budget": st["tiles_fallback_budget"],
                "tiles_fallback_minified": st["tiles_fallback_minified"]}
    for tname in ("fp16", "fp8"):
        a, b = runs.get(f"{tname}_mask"), runs.get(f"{tname}_4tap")
        if a and b:
            runs[f"{tname}_mask_vs_4tap"] = a["pixels_per_s"] / b["pixels_per_s"]
    ms = _timed_views(lambda: _ctf.ctf_filter(exact, uv, jac, cov, W, H, 0, "mask", 0, opts11, out, ev,
                                             stream=stream), k, 2, flush, stream)
    runs["exact_mask"] = {"pixels_per_s": npix / (ms / k * 1e-3), "ms_per_view": ms / k}
    res["filter_3840x2160"] = runs
    # FP64 oracle on a band of 16 rows of the same view (its own frame on both sides)
    band = slice(1000, 1016)
    buv, bjac, bcov = (np.ascontiguousarray(a[band]) for a in (sc.uv, sc.jac, sc.coverage))
    d_buv, d_bjac, d_bcov = (torch.from_numpy(a).to(dev) for a in (buv, bjac, bcov))
    bout = torch.empty((16, W, 4), device=dev)
    bev = torch.empty((16, W), dtype=torch.uint8, device=dev)
    orc = {}
    for tname in ("fp16", "fp8"):
        st_ = _ctf.ctf_mlp_export(texs[tname], ((1024, 1024, 8), (512, 512, 8)))
        if tname == "fp16":
            w = [st_["w1"], st_["w2"], st_["w3"]]
        else:
            w = [st_["ws0"][:, None] * st_["w1"] / st_["as0"][None, :],
                 st_["ws1"][:, None] * st_["w2"] / st_["as1"][None, :],
                 st_["ws2"][:, None] * st_["w3"] / st_["as2"][None, :]]
        mlp = oracle.MLP((st_["lat0"], st_["lat1"]), w[0].astype(np.float64), st_["b1"], w[1].astype(np.float64),
                         st_["b2"], w[2].astype(np.float64), st_["b3"])
        _ctf.ctf_filter(texs[tname], d_buv, d_bjac, d_bcov, W, 16, 0, "mask", 0, opts11, bout, bev, stream=stream)
        _ctf.ctf_sync_check(stream)
        t0 = time.perf_counter()
        ref, ref_ev, _ = oracle.filter_frame_learned_f64(mlp, 4096, 4096, buv, bjac, bcov, alg=oracle.ALG_MASK,
                                                         mask_dim=11)
        el = time.perf_counter() - t0
        g = bout.cpu().numpy().astype(np.float64)
        err = np.abs(g - ref)
        mse = float(np.mean(err[..., :3] ** 2))
        orc[tname] = {"rows": "1000..1015 of 2160", "pixels": 16 * W, "max_abs": float(err.max()),
                      "psnr_db": -10 * math.log10(max(mse, 1e-30)),
                      "counts_equal": bool(np.array_equal(bev.cpu().numpy(), ref_ev)), "oracle_s": el}
    res["vs_fp64_oracle_mask11"] = orc
    res["_textures"] = (exact, texs, blocks)
    _ctf.ctf_trainer_destroy(tr)
    return res


def bench_batch(args, dev, stream, learned_tex, block_tex):
    """Two view sets, each a list of tilted planes with their own
    magnification range inside [0.25, 64] and textures alternating a 2048^2
    block texture and the learned 4096^2 FP16 texture: 64 views of sizes
    uniform in [256, 3840] x [256, 2160], and 256 small views of sizes
    uniform in [64, 512]^2.  Each set: one autotuned batch (its own launch
    for every view of at least solo_tiles warp tiles, one persistent launch
    per kind for the rest) replayed from a CUDA graph against sequential
    ctf_filter calls."""
    out = _bench_batch_set(args, dev, stream, learned_tex, block_tex, 64, {})
    out["small_views"] = _bench_batch_set(args, dev, stream, learned_tex, block_tex, 256,
                                          {"min_w": 64, "min_h": 64, "max_w": 512, "max_h": 512})
    return out


def _bench_batch_set(args, dev, stream, learned_tex, block_tex, n_views, sizes):
    import torch
    from paper_2506_17770_gb300 import _ctf, synth
    t0 = time.perf_counter()
    tex_sizes = ((2048, 2048), (4096, 4096)) if learned_tex is not None else ((2048, 2048),)
    raw = synth.uneven_views(n_views, textures=tex_sizes, **sizes)
    gen_s = time.perf_counter() - t0
    views = []
    npix = 0
    for i, (sc, ti) in enumerate(raw):
        tex = block_tex if ti == 0 else learned_tex
        views.append({"tex": tex, "uv": torch.from_numpy(sc.uv).to(dev), "jac": torch.from_numpy(sc.jac).to(dev),
                      "coverage": torch.from_numpy(sc.coverage).to(dev), "width": sc.W, "height": sc.H,
                      "view_id": i, "out_rgba": torch.empty((sc.H, sc.W, 4), device=dev),
                      "out_evals": torch.empty((sc.H, sc.W), dtype=torch.uint8, device=dev)})
        npix += sc.W * sc.H
    alg = "mask"
    best, tune_ms = _ctf.ctf_batch_autotune(views, alg, 0, _ctf.batch_opts(mask_dim=11), stream=stream)
    g = _ctf.ctf_batch_graph_create(views, alg, 0, best)
    k = max(3, min(args.steps, 10))
    ms_graph = _timed_views(lambda: _ctf.ctf_batch_graph_launch(g, stream=stream), k, 2, None, stream)
    fo = {"tile_w": best.filter.tile_w, "tile_h": best.filter.tile_h, "mask_dim": 11}
    tw, th = best.filter.tile_w, best.filter.tile_h
    n_solo = sum(1 for v in views if best.solo_tiles > 0 and
                 ((v["width"] + tw - 1) // tw) * ((v["height"] + th - 1) // th) >= best.solo_tiles)

    def sequential():
        for v in views:
            _ctf.ctf_filter(v["tex"], v["uv"], v["jac"], v["coverage"], v["width"], v["height"], v["view_id"], alg, 0,
                            fo, v["out_rgba"], v["out_evals"], stream=stream)

    ms_seq = _timed_views(sequential, k, 2, None, stream)
    st = _ctf.ctf_filter_batch(views, alg, 0, best, stats=True, stream=stream)
    _ctf.ctf_sync_check(stream)
    _ctf.ctf_batch_graph_destroy(g)
    tg, ts = ms_graph / k * 1e-3, ms_seq / k * 1e-3

    # each kind of texel evaluation on its own (same configuration)
    kinds = {}
    for name, sub in (("block_views", [v for v in views if v["tex"] is block_tex]),
                      ("learned_views", [v for v in views if v["tex"] is not block_tex])):
        if not sub:
            continue
        gs = _ctf.ctf_batch_graph_create(sub, alg, 0, best)
        ms_g = _timed_views(lambda: _ctf.ctf_batch_graph_launch(gs, stream=stream), k, 2, None, stream)
        _ctf.ctf_batch_graph_destroy(gs)

        def seq_sub(sub=sub):
            for v in sub:
                _ctf.ctf_filter(v["tex"], v["uv"], v["jac"], v["coverage"], v["width"], v["height"], v["view_id"],
                                alg, 0, fo, v["out_rgba"], v["out_evals"], stream=stream)

        ms_s = _timed_views(seq_sub, k, 2, None, stream)
        px = sum(v["width"] * v["height"] for v in sub)
        kinds[name] = {"views": len(sub), "pixels": px, "graph_ms": ms_g / k, "sequential_ms": ms_s / k,
                       "graph_vs_sequential": ms_s / ms_g}
    return {"views": len(views), "sizes": sizes or {"min_w": 256, "min_h": 256, "max_w": 3840, "max_h": 2160},
            "pixels": npix, "input_gen_s": gen_s,
            "textures": "2048^2 block / 4096^2 learned FP16 alternating" if learned_tex is not None else "2048^2 block",
            "algorithm": "mask11+stf", "autotuned": best.as_dict(), "autotune_best_ms": tune_ms,
            "solo_views": n_solo,
            "graph_pixels_per_s": npix / tg, "graph_ms": tg * 1e3,
            "sequential_pixels_per_s": npix / ts, "sequential_ms": ts * 1e3, "graph_vs_sequential": ts / tg,
            "evals_per_pixel": st["texel_evals"] / max(1, st["pixels_active"]), "by_kind": kinds,
            "l2": f"not flushed: {npix * 42 / 1e6:.0f} MB of pixel I/O per pass, above the 129 MB L2"}


def max_over_ranks(x, device):
    """The largest of the ranks' values (the slowest rank's time per step),
    returned on every rank (NCCL tensors on the GPU, gloo ones on the CPU)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, npix_per_rank, ms_per_step):
    """Whole-job pixels/s: every rank filters its own view of npix_per_rank
    pixels per step (no exchange between ranks), the job as slow as its
    slowest rank."""
    return world * npix_per_rank / (ms_per_step * 1e-3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reference_arm(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    sc, blocks, Wt, Ht, desc = workload(args.workload, 0)
    alg, opts = HEADLINE
    npix = sc.W * sc.H
    for _ in range(max(args.warmup, 0)):
        run_cpu_oracle(sc, blocks, Wt, Ht, alg, opts, 0.0, 1)
    t0 = time.perf_counter()
    ev = 0
    for _ in range(args.steps):
        _, _, e = run_cpu_oracle(sc, blocks, Wt, Ht, alg, opts, 0.0, 1)
        ev += e
    el = time.perf_counter() - t0
    value = npix * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pixels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc}", "algorithm": "mask11+stf", "tile": "8x4",
                       "l2": "n/a (CPU)"},
            "evals_per_pixel": ev / (npix * args.steps),
            "cpu_baseline": {"value": value, "unit": "pixels/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full views, single thread"},
            "e2e": {"value": value, "unit": "pixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def ours_arm(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    from paper_2506_17770_gb300 import _ctf, build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    _ctf.load()

    sc, blocks, Wt, Ht, desc = workload(args.workload, rank)
    W, H = sc.W, sc.H
    npix = W * H
    dev = torch.device("cuda", torch.cuda.current_device())
    uv = torch.from_numpy(sc.uv).to(dev)
    jac = torch.from_numpy(sc.jac).to(dev)
    cov = torch.from_numpy(sc.coverage).to(dev) if sc.coverage is not None else None
    out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    ev = torch.empty((H, W), dtype=torch.uint8, device=dev)
    tex = _ctf.ctf_texture_create(Wt, Ht, blocks)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    tex_bytes = blocks.nbytes

    def launch(alg, opts):
        _ctf.ctf_filter(tex, uv, jac, cov, W, H, rank, alg, 0, opts, out, ev, stream=stream)

    def timed(alg, opts, steps, warmup, barrier=False):
        for _ in range(warmup):
            flush()
            launch(alg, opts)
        torch.cuda.synchronize()
        if barrier and world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        w0 = time.perf_counter()
        for i in range(steps):
            flush()
            starts[i].record(stream)
            launch(alg, opts)
            ends[i].record(stream)
        torch.cuda.synchronize()
        if barrier and world > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - w0
        ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
        return ms, wall

    def stats_of(alg, opts):
        return _ctf.ctf_filter(tex, uv, jac, cov, W, H, rank, alg, 0, opts, out, ev, stats=True, stream=stream)

    alg, opts = HEADLINE
    clocks = ClockSampler(local)
    clocks.start()
    ms, wall = timed(alg, opts, args.steps, args.warmup, barrier=True)
    clk = clocks.stop()
    ms_per_step = ms / args.steps
    if world > 1:
        ms_per_step = max_over_ranks(ms_per_step, dev)
    st = stats_of(alg, opts)
    value = weak_scaling_value(world, npix, ms_per_step)
    evpp = st["texel_evals"] / max(1, st["pixels_active"])

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return 0

    # --- side measurements (rank 0 only) ---
    extras = {}
    if not args.no_extras:
        k = min(args.steps, 1000)
        ref4 = ref16 = None
        for key, a, o in [("mask11", HEADLINE[0], {})] + OTHERS:
            oo = dict(HEADLINE[1])
            oo.update(o)
            if key == "mask11":  # headline image, for the error against 4-tap only
                stats_of(a, oo)
                img = out.clone()
                continue
            ms_a, _ = timed(a, oo, k, 5)
            sa = stats_of(a, oo)
            if key == "4tap":
                ref4 = out.clone()
                extras["mask11"] = {"psnr_vs_4tap_db": _psnr(img, ref4)}
            if key.endswith("_16tap"):
                ref16 = out.clone()
            extras[key] = {"pixels_per_s": npix / (ms_a / k * 1e-3), "ms_per_view": ms_a / k,
                           "evals_per_pixel": sa["texel_evals"] / max(1, sa["pixels_active"]),
                           "tiles_success": sa["tiles_success"], "tiles_fallback_budget": sa["tiles_fallback_budget"],
                           "tiles_fallback_minified": sa["tiles_fallback_minified"],
                           "achieved_gbs": algorithmic_bytes(a, npix, tex_bytes, cov is not None) / (ms_a / k * 1e-3) / 1e9}
            if key.endswith("_mask16"):
                extras[key]["psnr_vs_16tap_db"] = _psnr(out, ref16)
            elif ref4 is not None and key != "4tap" and not key.endswith("_16tap"):
                extras[key]["psnr_vs_4tap_db"] = _psnr(out, ref4)
    # end-to-end through the host entry point (pinned host buffers).  Three
    # sets of buffers in turn (3 x 87 MB, above the 129 MB L2), so that no
    # step finds the previous step's inputs in L2.
    sets = []
    for _ in range(3):
        sets.append((torch.from_numpy(sc.uv).pin_memory(), torch.from_numpy(sc.jac).pin_memory(),
                     torch.from_numpy(sc.coverage).pin_memory() if sc.coverage is not None else None,
                     torch.empty((H, W, 4), dtype=torch.float32).pin_memory(),
                     torch.empty((H, W), dtype=torch.uint8).pin_memory()))
    h_cov = sets[0][2]
    k_e2e = max(3, min(args.steps, 200))
    for i in range(3):
        h_uv, h_jac, h_c, h_out, h_ev = sets[i % 3]
        _ctf.ctf_filter_host(tex, h_uv, h_jac, h_c, W, H, 0, alg, 0, opts, h_out, h_ev, stream=stream)
    t0 = time.perf_counter()
    for i in range(k_e2e):
        h_uv, h_jac, h_c, h_out, h_ev = sets[i % 3]
        _ctf.ctf_filter_host(tex, h_uv, h_jac, h_c, W, H, 0, alg, 0, opts, h_out, h_ev, stream=stream)
    e2e_s = (time.perf_counter() - t0) / k_e2e
    h2d = npix * (8 + 16 + (1 if h_cov is not None else 0))
    d2h = npix * (16 + 1)

    peak, peak_kind = measured_peaks()
    learned = None
    batch = None
    if not args.no_extras and not args.no_learned:
        learned = bench_learned(args, dev, stream, flush, {"bf16": measured_bf16()[0], "bf16_kind": measured_bf16()[1]})
    if not args.no_extras and not args.no_batch:
        ltex = learned["_textures"][1]["fp16"] if learned else None
        batch = bench_batch(args, dev, stream, ltex, tex)
    if learned:
        exact_l, texs_l, _ = learned.pop("_textures")
        for t in list(texs_l.values()) + [exact_l]:
            _ctf.ctf_texture_destroy(t)
    abytes = algorithmic_bytes(alg, npix, tex_bytes, cov is not None)
    achieved = abytes / (ms_per_step * 1e-3) / 1e9
    traffic = ncu_traffic(args.workload, "mask11")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": abytes,
                "kernel": "exact_filter_kernel<MASK, 8x4, 11>"}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        frames, el, evs = run_cpu_oracle(sc, blocks, Wt, Ht, alg, opts, seconds=10.0)
        cpu = {"value": frames * npix / el, "unit": "pixels/s", "cores": 1, "kind": "oracle",
               "sample": f"{frames} full {W}x{H} views of the same workload, mask11+stf, single thread, "
                         f"{el:.1f} s"}

    fourtap = extras.get("4tap")
    line = {"metric": METRIC, "value": value, "unit": "pixels/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc}", "algorithm": "mask11+stf", "tile": "8x4",
                       "budget": 32, "views_per_step": world, "l2": "flushed before every step (256 MiB write, then 256 MiB read)"},
            "evals_per_pixel": evpp,
            "texel_evals_per_s": value * evpp,
            "vs_4tap": (value / world) / fourtap["pixels_per_s"] if fourtap else None,
            "algorithms": extras,
            "stats": st,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": npix / e2e_s, "unit": "pixels/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "entry_point": "ctf_filter_host",
                    "transfer": "page-locked host buffers: inputs read and the image written in place by the kernel "
                                "over NVLink-C2C, the counts copied back in one copy; three buffer sets in turn "
                                "(261 MB, above L2)"},
            "learned": learned,
            "batch": batch,
            "gpu_launches": args.steps,
            "clocks": clk,
            "wall_s_timed_region": wall}
    print(json.dumps(line), flush=True)
    _ctf.ctf_texture_destroy(tex)
    if world > 1:
        torch.distributed.barrier()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
