#!/usr/bin/env python3
"""Throughput of collaborative texture filtering on one GB300 (or N, one
process per GPU, each filtering its own view: weak scaling, no collective on
the data path).

Headline workload (default "learned2160", the costly-evaluation case of the
paper's Sec. 4.3.1): a 4096x4096 procedural RGBA texture (6 octaves of
gradient noise plus checker edges), block-encoded, learned by the library's
own trainer into two latent grids (1024^2 and 512^2, 8 FP16 channels) and a
16-64-64-4 MLP from 64M texels of its exact decode; then a 3840x2160 view of
a tilted plane with magnification log-uniform in [1, 16], filtered with the
learned FP16 decode on the tcgen05 tensor cores by Mask Sampling (11x11 mask,
one-tap STF fallback, 8x4 warps).  A step filters the whole view.

Beside the headline (rank 0, in the same JSON line):
  * every algorithm on the learned view in FP16 and FP8, the speedup over
    per-pixel 4-tap, and the error against the FP64 oracle on a row band;
  * the exact block-decode workload "frame1080" (1920x1080 perspective ground
    plane plus 3 tilted quads, 2048^2 random blocks) with its own HBM
    roofline, CPU baseline and end-to-end figure;
  * 64 and 256 uneven views in one persistent graph-captured batch.

Timing: W warm-up steps, then K timed steps; before every step a 256 MiB
buffer is written to flush L2 and a second 256 MiB buffer is read, so that L2
holds clean lines; each step's kernel is timed with CUDA events on the
launching stream.  One JSON line on rank 0.

CPU baselines: the FP64 (learned) or FP32 (exact) oracle, plain C, timed on
the host's cores, once on one thread over a band of rows and once over the
whole view with one process per core (row bands of whole tile rows; the
oracle gives each band the image it has inside the whole view).

--impl reference times that oracle alone on the same workload over all host
cores: each step is the whole view.  For the learned workload it runs with
seeded random parameters of the same network (the oracle's cost does not
depend on their values, and the reference arm uses no GPU to train them).
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
import tempfile
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
FALLBACK_BF16_TFLOPS = 1900.0
MLP_FLOP_PER_EVAL = 2 * (16 * 64 + 64 * 64 + 64 * 4)  # 10,752
LEARNED_TEX = 4096
LEARNED_LATENTS = ((1024, 1024), (512, 512))
LEARNED_VIEW = (3840, 2160, 1.0, 16.0)   # W, H, magnification range
WORKLOADS = ("learned2160", "frame1080", "frame2160", "plane128")


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=WORKLOADS, default="learned2160")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline only (for profiling)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-views workload")
    ap.add_argument("--train-steps", type=int, default=8192, help="training steps (learned)")
    ap.add_argument("--train-batch", type=int, default=8192, help="texels per training step (learned)")
    return ap.parse_args(argv)


def workload(name: str, rank: int):
    """Exact-decode workloads: (scene, blocks, Wt, Ht, description)."""
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


def learned_scene(rank: int):
    from paper_2506_17770_gb300 import synth
    W, H, lo, hi = LEARNED_VIEW
    return synth.perspective_view(W, H, LEARNED_TEX, LEARNED_TEX, lo, hi, seed=synth.SEED_SCENE + rank)


def learned_config():
    W, H, lo, hi = LEARNED_VIEW
    return {"workload": f"learned2160: {W}x{H} tilted plane, magnification log-uniform in [{lo:g}, {hi:g}], "
                        f"learned decode of a {LEARNED_TEX}x{LEARNED_TEX} procedural texture (latent grids "
                        f"1024^2 + 512^2 x 8 FP16, MLP 16-64-64-4)",
            "algorithm": "mask11+stf", "tile": "8x4", "budget": 32,
            "l2": "view inputs 207 MB, above the 129 MB L2; the GPU arm also flushes L2 before every step"}


def exact_config(name, desc):
    return {"workload": f"{name}: {desc}", "algorithm": "mask11+stf", "tile": "8x4", "budget": 32,
            "l2": "flushed before every GPU step (256 MiB write, then 256 MiB read)"}


def algorithmic_bytes(alg: str, npix: int, tex_bytes: int, has_cov: bool) -> int:
    """Bytes a kernel must move: per pixel uv 8 + (jac 16 for the collaborative
    algorithms, which vote on minification) + coverage 1 + RGBA32F 16 + count 1,
    plus the texture read once."""
    per = 8 + 16 + 1 + (1 if has_cov else 0)
    if alg not in ("4tap", "stf"):
        per += 16
    return npix * per + tex_bytes


def _peaks_file():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return None


def measured_peaks():
    d = _peaks_file()
    if d and "hbm_gbs" in d:
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def measured_bf16():
    d = _peaks_file()
    if d and "bf16_tflops" in d:
        return float(d["bf16_tflops"]), "measured burst bf16 (fp16 runs at the bf16 rate)"
    return FALLBACK_BF16_TFLOPS, "fallback"


def kernel_source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2506_17770_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


EXACT_SOURCES = ("ctf_filter.cu", "ctf_device.cuh", "ctf_exact_tile.cuh", "ctf_select.cuh")
LEARNED_SOURCES = ("ctf_mlp_ws2.cu", "ctf_mlp_chain.cuh", "ctf_mlp.cuh", "ctf_device.cuh", "ctf_select.cuh",
                   "tc_ops.cuh")


def ncu_traffic(key: str, sources):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(key)
    if not e or e.get("source_hash") != kernel_source_hash(sources):
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


def timed_steps(launch, steps, warmup, flush, stream, world):
    """The contract's timed region: W warm-up steps, then K steps bracketed
    by a barrier and a synchronize on both sides; each step's launch timed
    with CUDA events on its stream after an L2 flush.  Returns the summed
    event time (ms) and the wall time of the region (s)."""
    import torch
    for _ in range(warmup):
        flush()
        launch()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    w0 = time.perf_counter()
    for i in range(steps):
        flush()
        starts[i].record(stream)
        launch()
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - w0
    return sum(s.elapsed_time(e) for s, e in zip(starts, ends)), wall


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


# ---------------------------------------------------------------------------
# The CPU oracle on the host's cores (test infrastructure: only this file's
# CPU legs run it, never the GPU path)
# ---------------------------------------------------------------------------
_POOL = {}


def _pool_init(folder):
    """Worker set-up: memory-map the view and the texture parameters."""
    import numpy as np
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    st = {}
    for f in os.listdir(folder):
        if f.endswith(".npy"):
            st[f[:-4]] = np.load(os.path.join(folder, f), mmap_mode="r")
    with open(os.path.join(folder, "meta.json")) as fh:
        st["meta"] = json.load(fh)
    if "lat0" in st:
        st["mlp"] = oracle.MLP((st["lat0"], st["lat1"]), st["w1"], st["b1"], st["w2"], st["b2"], st["w3"], st["b3"])
    _POOL.clear()
    _POOL.update(st)


def _pool_band(rows):
    """Filter rows [y0, y1) of the view with the oracle, as the band of the
    view it is; returns (texel evaluations, active pixels, seconds)."""
    import numpy as np
    import oracle
    y0, y1 = rows
    s = _POOL
    m = s["meta"]
    uv = np.ascontiguousarray(s["uv"][y0:y1])
    jac = np.ascontiguousarray(s["jac"][y0:y1])
    cov = np.ascontiguousarray(s["cov"][y0:y1]) if "cov" in s else None
    kw = dict(alg=ALG_ID[m["alg"]], mask_dim=m["mask_dim"], tile_w=8, tile_h=4, budget=32, y_offset=y0)
    t0 = time.perf_counter()
    if "mlp" in s:
        _, _, st = oracle.filter_frame_learned_f64(s["mlp"], m["Wt"], m["Ht"], uv, jac, cov, **kw)
    else:
        _, _, st = oracle.filter_frame(s["blocks"], m["Wt"], m["Ht"], uv, jac, cov, **kw)
    return st["texel_evals"], st["pixels_active"], time.perf_counter() - t0


class OraclePool:
    """The oracle over the whole view, one process per host core (spawned,
    never forked from a process that has used the GPU), each taking bands of
    16 rows; and the same oracle on one thread in this process."""

    BAND = 16

    def __init__(self, arrays: dict, meta: dict, cores: int):
        import multiprocessing as mp
        import numpy as np
        self.dir = tempfile.mkdtemp(prefix="ctf_oracle_pool_")
        for k, v in arrays.items():
            np.save(os.path.join(self.dir, k + ".npy"), np.ascontiguousarray(v))
        with open(os.path.join(self.dir, "meta.json"), "w") as fh:
            json.dump(meta, fh)
        self.H = int(arrays["uv"].shape[0])
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores, initializer=_pool_init, initargs=(self.dir,))
        # every worker set up (and warm) before anything is timed
        self.pool.map(_pool_band, [(0, min(4, self.H))] * (2 * cores), chunksize=1)

    def bands(self, stride=1):
        b = [(y, min(y + self.BAND, self.H)) for y in range(0, self.H, self.BAND)]
        return b[::stride]

    def all_cores(self, views=1):
        """(seconds, texel evaluations, active pixels) of `views` passes over
        the whole view."""
        t0 = time.perf_counter()
        res = self.pool.map(_pool_band, self.bands() * views, chunksize=1)
        el = time.perf_counter() - t0
        return el, sum(r[0] for r in res), sum(r[1] for r in res)

    def one_thread(self, stride):
        """(seconds, pixels) of every `stride`-th band on one thread (this
        process), a sample that spans the view's magnification range."""
        _pool_init(self.dir)
        b = self.bands(stride)
        t0 = time.perf_counter()
        for rows in b:
            _pool_band(rows)
        el = time.perf_counter() - t0
        W = int(_POOL["uv"].shape[1])
        _POOL.clear()
        return el, sum((y1 - y0) * W for y0, y1 in b)

    def close(self):
        import shutil
        self.pool.close()
        self.pool.join()
        shutil.rmtree(self.dir, ignore_errors=True)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(arrays, meta, stride=8, views=1, what=""):
    """The oracle's pixels/s on the host's cores (all of them, the reported
    value: `views` passes over the whole view) and on one thread (a sample of
    every `stride`-th band)."""
    cores = host_cores()
    pool = OraclePool(arrays, meta, cores)
    try:
        el, evs, act = pool.all_cores(views)
        st_s, st_px = pool.one_thread(stride)
    finally:
        pool.close()
    H, W = arrays["uv"].shape[:2]
    return {"value": views * W * H / el, "unit": "pixels/s", "cores": cores, "kind": "oracle",
            "sample": f"{views} pass{'es' if views > 1 else ''} over the whole {W}x{H} view {what}in bands of "
                      f"16 rows, one process per host core ({cores}), {el:.2f} s",
            "single_thread": {"value": st_px / st_s, "unit": "pixels/s", "cores": 1,
                              "sample": f"one band of 16 rows in every {stride} ({st_px} pixels), {st_s:.2f} s"},
            "texel_evals_per_pixel": evs / max(1, act)}


# ---------------------------------------------------------------------------
# Learned decode: texture, training, textures of both precisions
# ---------------------------------------------------------------------------
def learned_textures(args, dev, stream):
    """The 4096^2 procedural target, block-encoded; the library's trainer
    learns it from texels of its exact decode (`--train-steps` x
    `--train-batch` texels, 8192 x 8192 = 64M by default); exported FP16 and
    FP8 textures and their texel error against the exact decode."""
    import torch
    from paper_2506_17770_gb300 import _ctf, synth
    info = {}
    t0 = time.perf_counter()
    rgba = synth.procedural_rgba8(LEARNED_TEX, device=dev)
    blocks = synth.encode_blocks(rgba)
    info["input_gen_s"] = time.perf_counter() - t0
    exact = _ctf.ctf_texture_create(LEARNED_TEX, LEARNED_TEX, blocks)
    steps, batch = args.train_steps, args.train_batch
    desc = _ctf.train_desc(LEARNED_LATENTS, batch=batch, total_steps=steps, lr_weights=1e-2, lr_latents=1e-1,
                           lr_final_frac=0.02, seed=3)
    tr = _ctf.ctf_trainer_create(exact, desc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _ctf.ctf_trainer_step(tr, steps, stream=stream)
    _ctf.ctf_sync_check(stream)
    train_s = time.perf_counter() - t0
    info["training"] = {"steps": steps, "batch": batch, "texels": steps * batch, "seconds": train_s,
                        "texels_per_s": steps * batch / train_s,
                        "schedule": "Adam, lr 1e-2 (weights) / 1e-1 (latents), linear decay to 2% over all steps"}
    texs = {"fp16": _ctf.ctf_trainer_export(tr, _ctf.CTF_EVAL_MLP_FP16),
            "fp8": _ctf.ctf_trainer_export(tr, _ctf.CTF_EVAL_MLP_FP8)}
    _ctf.ctf_trainer_destroy(tr)
    for k, t in texs.items():
        mse, mx = _ctf.ctf_texture_compare(exact, t, stream=stream)
        info[f"{k}_texels_vs_exact"] = {"psnr_db": -10 * math.log10(max(mse, 1e-30)), "max_abs": mx}
    return exact, texs, info


def oracle_mlp_arrays(tex, tname):
    """The stored parameters of a learned texture as the FP64 oracle takes
    them: FP16 values as they are; FP8 weights times their output-channel
    scale over the input's activation scale (the effective weights)."""
    from paper_2506_17770_gb300 import _ctf
    st = _ctf.ctf_mlp_export(tex, tuple(tuple(s) + (8,) for s in LEARNED_LATENTS))
    if tname == "fp16":
        w = [st["w1"], st["w2"], st["w3"]]
    else:
        w = [st["ws0"][:, None] * st["w1"] / st["as0"][None, :],
             st["ws1"][:, None] * st["w2"] / st["as1"][None, :],
             st["ws2"][:, None] * st["w3"] / st["as2"][None, :]]
    return {"lat0": st["lat0"], "lat1": st["lat1"], "w1": w[0], "b1": st["b1"], "w2": w[1], "b2": st["b2"],
            "w3": w[2], "b3": st["b3"]}


def random_mlp_arrays(seed=3):
    """Seeded random parameters of the learned decode's network."""
    import numpy as np
    g = np.random.default_rng(seed)
    (w0, h0), (w1_, h1_) = LEARNED_LATENTS
    return {"lat0": g.normal(0, 1.0, (h0, w0, 8)).astype(np.float16).astype(np.float32),
            "lat1": g.normal(0, 1.0, (h1_, w1_, 8)).astype(np.float16).astype(np.float32),
            "w1": g.normal(0, 0.35, (64, 16)), "b1": g.normal(0, 0.1, 64), "w2": g.normal(0, 0.18, (64, 64)),
            "b2": g.normal(0, 0.1, 64), "w3": g.normal(0, 0.04, (4, 64)), "b3": np.array([0.5, 0.5, 0.5, 0.9])}


def learned_others(args, dev, stream, flush, sc, texs, exact, peak_tf, peak_kind):
    """Every algorithm on the learned view, FP16 and FP8, against exact 4-tap
    and (on a row band) against the FP64 oracle."""
    import numpy as np
    import torch
    import oracle
    from paper_2506_17770_gb300 import _ctf
    W, H = sc.W, sc.H
    npix = W * H
    uv, jac, cov = (torch.from_numpy(a).to(dev) for a in (sc.uv, sc.jac, sc.coverage))
    out = torch.empty((H, W, 4), device=dev)
    ev = torch.empty((H, W), dtype=torch.uint8, device=dev)
    ref_exact = torch.empty((H, W, 4), device=dev)
    _ctf.ctf_filter(exact, uv, jac, cov, W, H, 0, "4tap", 0, None, ref_exact, ev, stream=stream)
    k = max(3, min(args.steps, 20))
    runs = {}
    ref4 = {}
    opts11 = {"mask_dim": 11}
    for tname in ("fp16", "fp8"):
        tex = texs[tname]
        for name in ("4tap", "stf", "mask", "mask_group_dedup", "box", "list_merge", "mask_fallback_cplus",
                     "mask_two_texels_per_lane"):
            if tname == "fp8" and name in ("stf", "box", "list_merge"):
                continue
            alg = "mask" if name.startswith("mask") else name
            o = {"mask": opts11, "mask_group_dedup": {"mask_dim": 11, "group_dedup": 1},
                 "mask_fallback_cplus": {"mask_dim": 11, "fallback": 2},
                 "mask_two_texels_per_lane": {"mask_dim": 11, "texels_per_lane": 2, "budget": 64}}.get(name)
            ms = _timed_views(lambda: _ctf.ctf_filter(tex, uv, jac, cov, W, H, 0, alg, 0, o, out, ev,
                                                     stream=stream), k, 2, flush, stream)
            st = _ctf.ctf_filter(tex, uv, jac, cov, W, H, 0, alg, 0, o, out, ev, stats=True, stream=stream)
            _ctf.ctf_sync_check(stream)
            mse = torch.mean((out[..., :3] - ref_exact[..., :3]) ** 2).item()
            if name == "4tap":
                ref4[tname] = out.clone()
            t = ms / k * 1e-3
            flops = st["texel_evals_unique"] * MLP_FLOP_PER_EVAL  # evaluations done
            peak = peak_tf * (2.0 if tname == "fp8" else 1.0)
            runs[f"{tname}_{name}"] = {
                "pixels_per_s": npix / t, "ms_per_view": t * 1e3, "us_per_mpixel": t * 1e6 / (npix / 1e6),
                "evals_per_pixel": st["texel_evals"] / max(1, st["pixels_active"]),
                "evaluations_done_per_pixel": st["texel_evals_unique"] / max(1, st["pixels_active"]),
                "texel_evals_per_s": st["texel_evals"] / t,
                "psnr_vs_exact_4tap_db": -10 * math.log10(max(mse, 1e-30)),
                "psnr_vs_learned_4tap_db": (_psnr(out, ref4[tname]) if name != "4tap" else None),
                "tensor": {"achieved_tflops": flops / t / 1e12, "peak_tflops": peak,
                           "frac": flops / t / 1e12 / peak,
                           "peak_kind": peak_kind + (" x2 (nominal fp8/fp16 ratio)" if tname == "fp8" else "")},
                "tiles_success": st["tiles_success"], "tiles_fallback_budget": st["tiles_fallback_budget"],
                "tiles_fallback_minified": st["tiles_fallback_minified"]}
    for tname in ("fp16", "fp8"):
        a, b = runs.get(f"{tname}_mask"), runs.get(f"{tname}_4tap")
        if a and b:
            runs[f"{tname}_mask_vs_4tap"] = a["pixels_per_s"] / b["pixels_per_s"]
    ms = _timed_views(lambda: _ctf.ctf_filter(exact, uv, jac, cov, W, H, 0, "mask", 0, opts11, out, ev,
                                             stream=stream), k, 2, flush, stream)
    runs["exact_mask"] = {"pixels_per_s": npix / (ms / k * 1e-3), "ms_per_view": ms / k}
    # FP64 oracle on three bands of 16 rows (top, middle, bottom of the view)
    orc = {}
    for tname in ("fp16", "fp8"):
        a = oracle_mlp_arrays(texs[tname], tname)
        mlp = oracle.MLP((a["lat0"], a["lat1"]), a["w1"], a["b1"], a["w2"], a["b2"], a["w3"], a["b3"])
        errs, mses, equal, px = [], [], True, 0
        # the GPU image of the whole view against the oracle on three bands
        # of 16 rows, each filtered as the band of the view it is
        _ctf.ctf_filter(texs[tname], uv, jac, cov, W, H, 0, "mask", 0, opts11, out, ev, stream=stream)
        _ctf.ctf_sync_check(stream)
        for y0 in (0, H // 2 - (H // 2) % 4, H - 16):
            band = slice(y0, y0 + 16)
            buv, bjac, bcov = (np.ascontiguousarray(x[band]) for x in (sc.uv, sc.jac, sc.coverage))
            ref, ref_ev, _ = oracle.filter_frame_learned_f64(mlp, LEARNED_TEX, LEARNED_TEX, buv, bjac, bcov,
                                                             alg=oracle.ALG_MASK, mask_dim=11, y_offset=y0)
            g = out[band].cpu().numpy().astype(np.float64)
            err = np.abs(g - ref)
            errs.append(float(err.max()))
            mses.append(float(np.mean(err[..., :3] ** 2)))
            equal &= bool(np.array_equal(ev[band].cpu().numpy(), ref_ev))
            px += 16 * W
        mse = float(np.mean(mses))
        orc[tname] = {"rows": f"0..15, {H // 2 - (H // 2) % 4}.., {H - 16}..{H - 1} of {H}", "pixels": px,
                      "max_abs": max(errs), "psnr_db": -10 * math.log10(max(mse, 1e-30)), "counts_equal": equal}
    return {"filter_3840x2160": runs, "vs_fp64_oracle_mask11": orc}


def e2e_host(tex, sc, alg, opts, k, stream):
    """ctf_filter_host on page-locked host buffers: three buffer sets in turn
    (each above L2 at these sizes), so that no step finds the previous step's
    inputs in L2.  Returns (seconds per call, h2d bytes, d2h bytes)."""
    import torch
    from paper_2506_17770_gb300 import _ctf
    W, H = sc.W, sc.H
    sets = []
    for _ in range(3):
        sets.append((torch.from_numpy(sc.uv).pin_memory(), torch.from_numpy(sc.jac).pin_memory(),
                     torch.from_numpy(sc.coverage).pin_memory() if sc.coverage is not None else None,
                     torch.empty((H, W, 4), dtype=torch.float32).pin_memory(),
                     torch.empty((H, W), dtype=torch.uint8).pin_memory()))
    for i in range(3):
        h_uv, h_jac, h_c, h_out, h_ev = sets[i]
        _ctf.ctf_filter_host(tex, h_uv, h_jac, h_c, W, H, 0, alg, 0, opts, h_out, h_ev, stream=stream)
    t0 = time.perf_counter()
    for i in range(k):
        h_uv, h_jac, h_c, h_out, h_ev = sets[i % 3]
        _ctf.ctf_filter_host(tex, h_uv, h_jac, h_c, W, H, 0, alg, 0, opts, h_out, h_ev, stream=stream)
    s = (time.perf_counter() - t0) / k
    npix = W * H
    h2d = npix * (8 + (16 if alg not in ("4tap", "stf") else 0) + (1 if sc.coverage is not None else 0))
    d2h = npix * (16 + 1)
    del sets
    return s, h2d, d2h


def link_roof(h2d, d2h, s, reps=5):
    """The host link's rate for one step's bytes: h2d bytes copied from
    page-locked host memory to the device and d2h bytes back, on two streams
    at once (copy engines, CUDA events, best of reps), beside the rate the
    end-to-end call achieved for the same bytes in s seconds."""
    import torch
    h_in = torch.empty(h2d, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(d2h, dtype=torch.uint8).pin_memory()
    d_in = torch.empty(h2d, dtype=torch.uint8, device="cuda")
    d_out = torch.zeros(d2h, dtype=torch.uint8, device="cuda")
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream()
        e0.record(cur)
        for st, dst, src in ((s_in, d_in, h_in), (s_out, h_out, d_out)):
            st.wait_event(e0)
            with torch.cuda.stream(st):
                dst.copy_(src, non_blocking=True)
            done = torch.cuda.Event()
            done.record(st)
            cur.wait_event(done)
        e1.record(cur)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    link = (h2d + d2h) / best / 1e9
    achieved = (h2d + d2h) / s / 1e9
    return {"achieved_GBps": achieved, "link_GBps": link, "frac": achieved / link,
            "how": "copy engines, both directions at once on two streams, the step's h2d and d2h bytes"}


E2E_NOTE = ("page-locked host buffers: inputs read and the image written in place by the kernel over "
            "NVLink-C2C, the counts copied back in one copy; three buffer sets in turn (above L2)")


def exact_section(args, dev, stream, flush, name, rank, world, headline):
    """The exact block-decode workload: Mask-11 (timed as the contract's
    steps when it is the headline), every other algorithm, HBM roofline,
    end-to-end through ctf_filter_host and the oracle on the host's cores."""
    import torch
    from paper_2506_17770_gb300 import _ctf
    sc, blocks, Wt, Ht, desc = workload(name, rank)
    W, H = sc.W, sc.H
    npix = W * H
    uv, jac = torch.from_numpy(sc.uv).to(dev), torch.from_numpy(sc.jac).to(dev)
    cov = torch.from_numpy(sc.coverage).to(dev) if sc.coverage is not None else None
    out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    ev = torch.empty((H, W), dtype=torch.uint8, device=dev)
    tex = _ctf.ctf_texture_create(Wt, Ht, blocks)
    alg, opts = HEADLINE
    res = {"config": exact_config(name, desc)}

    def launch(a=alg, o=opts):
        _ctf.ctf_filter(tex, uv, jac, cov, W, H, rank, a, 0, o, out, ev, stream=stream)

    def stats_of(a, o):
        return _ctf.ctf_filter(tex, uv, jac, cov, W, H, rank, a, 0, o, out, ev, stats=True, stream=stream)

    if headline:
        clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        clocks.start()
        ms, wall = timed_steps(launch, args.steps, args.warmup, flush, stream, world)
        res["clocks"] = clocks.stop()
        res["wall_s_timed_region"] = wall
        res["steps"] = args.steps
    else:
        k = max(3, min(args.steps, 200))
        ms = _timed_views(launch, k, 5, flush, stream)
        res["steps"] = k
    res["ms_per_step"] = ms / res["steps"]
    st = stats_of(alg, opts)
    res["stats"] = st
    res["npix"] = npix
    res["evals_per_pixel"] = st["texel_evals"] / max(1, st["pixels_active"])
    if rank != 0:
        _ctf.ctf_texture_destroy(tex)
        return res
    extras = {}
    if not args.no_extras:
        k = max(3, min(args.steps, 200))
        stats_of(alg, opts)
        img = out.clone()
        ref4 = ref16 = None
        for key, a, o in OTHERS:
            oo = dict(opts)
            oo.update(o)
            ms_a = _timed_views(lambda: launch(a, oo), k, 5, flush, stream)
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
                           "achieved_gbs": algorithmic_bytes(a, npix, blocks.nbytes, cov is not None)
                           / (ms_a / k * 1e-3) / 1e9}
            if key.endswith("_mask16"):
                extras[key]["psnr_vs_16tap_db"] = _psnr(out, ref16)
            elif ref4 is not None and key != "4tap" and not key.endswith("_16tap"):
                extras[key]["psnr_vs_4tap_db"] = _psnr(out, ref4)
        res["vs_4tap"] = (npix / (res["ms_per_step"] * 1e-3)) / extras["4tap"]["pixels_per_s"]
    res["algorithms"] = extras
    peak, peak_kind = measured_peaks()
    abytes = algorithmic_bytes(alg, npix, blocks.nbytes, cov is not None)
    achieved = abytes / (res["ms_per_step"] * 1e-3) / 1e9
    res["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                       "traffic": ncu_traffic(f"{name}:mask11", EXACT_SOURCES), "peak_kind": peak_kind,
                       "algorithmic_bytes_per_launch": abytes, "kernel": "exact_filter_kernel<MASK, 8x4, 11>"}
    s, h2d, d2h = e2e_host(tex, sc, alg, opts, max(3, min(args.steps, 200)), stream)
    res["e2e"] = {"value": npix / s, "unit": "pixels/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                  "entry_point": "ctf_filter_host", "transfer": E2E_NOTE, "link": link_roof(h2d, d2h, s)}
    res["_tex"] = (tex, blocks)
    if not args.no_cpu_baseline and world == 1:
        arrays = {"uv": sc.uv, "jac": sc.jac, "blocks": blocks}
        if sc.coverage is not None:
            arrays["cov"] = sc.coverage
        res["cpu_baseline"] = cpu_baseline(arrays, {"alg": alg, "mask_dim": 11, "Wt": Wt, "Ht": Ht}, stride=2,
                                           views=max(1, 40 * 2073600 // npix),
                                           what="(FP32 oracle, Mask-11 + STF) ")
    return res


def learned_section(args, dev, stream, flush, rank, world):
    """The headline: learned FP16 decode, Mask-11 + STF on the 3840x2160
    view, timed as the contract's steps; tensor roofline, end-to-end through
    ctf_filter_host, the FP64 oracle on the host's cores."""
    import torch
    from paper_2506_17770_gb300 import _ctf
    exact, texs, info = learned_textures(args, dev, stream)
    sc = learned_scene(rank)
    W, H = sc.W, sc.H
    npix = W * H
    uv, jac, cov = (torch.from_numpy(a).to(dev) for a in (sc.uv, sc.jac, sc.coverage))
    out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    ev = torch.empty((H, W), dtype=torch.uint8, device=dev)
    tex = texs["fp16"]
    alg, opts = HEADLINE
    res = {"config": learned_config(), "training": info}

    def launch():
        _ctf.ctf_filter(tex, uv, jac, cov, W, H, rank, alg, 0, opts, out, ev, stream=stream)

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ms, wall = timed_steps(launch, args.steps, args.warmup, flush, stream, world)
    res["clocks"] = clocks.stop()
    res["wall_s_timed_region"] = wall
    res["steps"] = args.steps
    res["ms_per_step"] = ms / args.steps
    st = _ctf.ctf_filter(tex, uv, jac, cov, W, H, rank, alg, 0, opts, out, ev, stats=True, stream=stream)
    _ctf.ctf_sync_check(stream)
    res["stats"] = st
    res["npix"] = npix
    res["evals_per_pixel"] = st["texel_evals"] / max(1, st["pixels_active"])
    res["_textures"] = (exact, texs)
    if rank != 0:
        return res
    peak, peak_kind = measured_bf16()
    flop = st["texel_evals_unique"] * MLP_FLOP_PER_EVAL
    achieved = flop / (res["ms_per_step"] * 1e-3) / 1e12
    res["roofline"] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak,
                       "traffic": ncu_traffic("learned2160:fp16_mask11", LEARNED_SOURCES),
                       "peak_kind": peak_kind, "algorithmic_flop_per_launch": flop,
                       "flop_per_evaluation": MLP_FLOP_PER_EVAL,
                       "kernel": "mlp_filter_pf_kernel<MASK, 8x4, 11> (FP16 operands, FP32 accumulation in TMEM)"}
    # The same launch against the HBM roof: the per-pixel streams (uv, Jacobian,
    # coverage in; RGBA and count out) take longer at the measured copy rate
    # than the evaluations' FLOP at the tensor peak, so by the roofline model
    # this is the binding roof; the latents' lines are not counted.
    hbm_peak, hbm_kind = measured_peaks()
    pbytes = npix * (8 + 16 + (1 if cov is not None else 0) + 16 + 1)
    hbm_achieved = pbytes / (res["ms_per_step"] * 1e-3) / 1e9
    res["roofline_hbm"] = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                           "frac": hbm_achieved / hbm_peak, "peak_kind": hbm_kind,
                           "algorithmic_bytes_per_launch": pbytes,
                           "roof_us": {"hbm": pbytes / hbm_peak / 1e3, "tensor": flop / peak / 1e6}}
    if not args.no_extras:
        res["learned"] = learned_others(args, dev, stream, flush, sc, texs, exact, peak, peak_kind)
        f = res["learned"]["filter_3840x2160"]
        res["vs_4tap"] = (npix / (res["ms_per_step"] * 1e-3)) / f["fp16_4tap"]["pixels_per_s"]
    s, h2d, d2h = e2e_host(tex, sc, alg, opts, max(3, min(args.steps, 50)), stream)
    res["e2e"] = {"value": npix / s, "unit": "pixels/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                  "entry_point": "ctf_filter_host", "transfer": E2E_NOTE, "link": link_roof(h2d, d2h, s)}
    if not args.no_cpu_baseline and world == 1:
        arrays = {"uv": sc.uv, "jac": sc.jac, "cov": sc.coverage}
        arrays.update(oracle_mlp_arrays(tex, "fp16"))
        res["cpu_baseline"] = cpu_baseline(arrays, {"alg": alg, "mask_dim": 11, "Wt": LEARNED_TEX,
                                                    "Ht": LEARNED_TEX}, stride=8, views=1,
                                           what="(FP64 oracle of the learned decode with the FP16 texture's "
                                                "stored parameters, Mask-11 + STF) ")
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


def reference_arm(args):
    """The oracle alone, on the host's cores, on the headline workload: each
    step is one pass over the whole view, its bands spread over one process
    per core.  Only rank 0 runs; the other ranks exit without work."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    alg, opts = HEADLINE
    if args.workload == "learned2160":
        sc = learned_scene(0)
        arrays = {"uv": sc.uv, "jac": sc.jac, "cov": sc.coverage}
        arrays.update(random_mlp_arrays())
        meta = {"alg": alg, "mask_dim": 11, "Wt": LEARNED_TEX, "Ht": LEARNED_TEX}
        config, dtype = learned_config(), "f64"
        what = ("FP64 oracle of the learned decode (seeded random parameters of the same network; its cost does "
                "not depend on their values), Mask-11 + STF")
    else:
        sc, blocks, Wt, Ht, desc = workload(args.workload, 0)
        arrays = {"uv": sc.uv, "jac": sc.jac, "blocks": blocks}
        if sc.coverage is not None:
            arrays["cov"] = sc.coverage
        meta = {"alg": alg, "mask_dim": 11, "Wt": Wt, "Ht": Ht}
        config, dtype = exact_config(args.workload, desc), "f32"
        what = "FP32 oracle of the exact block decode, Mask-11 + STF"
    npix = sc.W * sc.H
    cores = host_cores()
    pool = OraclePool(arrays, meta, cores)
    try:
        for _ in range(max(args.warmup, 0)):
            pool.all_cores(1)
        t0 = time.perf_counter()
        evs = act = 0
        for _ in range(args.steps):
            _, e, a = pool.all_cores(1)
            evs += e
            act += a
        el = time.perf_counter() - t0
    finally:
        pool.close()
    value = npix * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pixels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": config,
            "evals_per_pixel": evs / max(1, act),
            "cpu_baseline": {"value": value, "unit": "pixels/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} passes over the whole {sc.W}x{sc.H} view ({what}), bands of "
                                       f"16 rows over one process per host core"},
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
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()

    learned = args.workload == "learned2160"
    if learned:
        head = learned_section(args, dev, stream, flush, rank, world)
        dtype = "f16"
    else:
        head = exact_section(args, dev, stream, flush, args.workload, rank, world, headline=True)
        dtype = "f32"
    ms_per_step = head["ms_per_step"]
    if world > 1:
        ms_per_step = max_over_ranks(ms_per_step, dev)
    value = weak_scaling_value(world, head["npix"], ms_per_step)
    evpp = head["evals_per_pixel"]
    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return 0

    exact = None
    if learned and not args.no_extras:
        exact = exact_section(args, dev, stream, flush, "frame1080", rank, 1, headline=False)
    batch = None
    if not args.no_extras and not args.no_batch:
        ltex = head["_textures"][1]["fp16"] if learned else None
        btex = (exact or head)["_tex"][0]
        batch = bench_batch(args, dev, stream, ltex, btex)
    for r in (head, exact):
        if r and "_tex" in r:
            _ctf.ctf_texture_destroy(r.pop("_tex")[0])
    if learned:
        ex, texs = head.pop("_textures")
        for t in list(texs.values()) + [ex]:
            _ctf.ctf_texture_destroy(t)

    line = {"metric": METRIC, "value": value, "unit": "pixels/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": head["config"],
            "evals_per_pixel": evpp, "texel_evals_per_s": value * evpp,
            "vs_4tap": head.get("vs_4tap"),
            "stats": head["stats"],
            "roofline": head["roofline"],
            "cpu_baseline": head.get("cpu_baseline"),
            "e2e": head["e2e"],
            "gpu_launches": args.steps,
            "clocks": head["clocks"],
            "wall_s_timed_region": head["wall_s_timed_region"]}
    if learned:
        line["dtype_note"] = ("FP16 operands with FP32 accumulation for the learned decode; FP32 coordinate "
                              "setup, selection and filter")
        line["training"] = head["training"]
        if "roofline_hbm" in head:
            line["roofline_hbm"] = head["roofline_hbm"]
        if "learned" in head:
            line["learned"] = head["learned"]
        if exact:
            exact.pop("_tex", None)
            line["exact_frame1080"] = {k: exact[k] for k in ("config", "ms_per_step", "evals_per_pixel", "vs_4tap",
                                                             "roofline", "e2e", "cpu_baseline", "algorithms",
                                                             "stats") if k in exact}
            line["exact_frame1080"]["pixels_per_s"] = exact["npix"] / (exact["ms_per_step"] * 1e-3)
    else:
        line["algorithms"] = head.get("algorithms")
    line["batch"] = batch
    print(json.dumps(line), flush=True)
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
