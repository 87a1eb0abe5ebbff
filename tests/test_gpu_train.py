"""GPU training of the learned decode: gradients against the FP64 oracle's
backward pass, what training gains, deterministic checkpoint/resume, and the
FP8 export against the FP64 oracle."""
import math
import os
import tempfile

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


def _decoded(blocks, Wt, Ht, xs, ys):
    return np.stack([oracle.decode_rgba8(blocks, Wt, Ht, int(x), int(y)) for x, y in zip(xs, ys)]) / 255.0


# The gradient kernel runs its products on the tensor cores with FP16
# operands (u = 2^-11 relative rounding each) and FP32 accumulation.  A
# gradient entry is a sum over texels of products along the chain
# features -> W1 -> H1 -> W2 -> H2 -> W3 -> e -> W3^T -> dH2 -> W2^T -> dH1
# -> W1^T, and every factor of such a product is rounded at most once on
# its way into an MMA, so |gpu - exact| <= K u G_abs entry by entry, with
# G_abs the same gradient computed from the absolute values of every factor
# and K the roundings on the longest path: 6 in the forward pass (F, W1,
# H1, W2, H2, W3), which reach the gradient through the error e, and 5 in
# the backward pass (e, W3^T, dH2, W2^T, dH1, with W1^T or the weight
# products' H1, F, H2 operands in place of the last), plus FP32
# accumulation (K 2^-24 with K <= 128 terms per MMA chain, below one more
# u).  The forward roundings enter through e, whose error is bounded by
# 6u Y_abs (Y_abs = |H2| |W3|^T + |b3|), so G_abs takes |e| + 6u Y_abs in
# place of |e|.  K = 12.  A ReLU unit whose input lies within the forward
# rounding of zero may switch, which moves an entry by a whole term rather
# than a fraction of it; such switches are rare and their terms small next
# to the largest entries, so the test takes the bound at the scale of the
# gradient: max |gpu - exact| <= K u max G_abs per parameter array.
FP16_U = 2.0 ** -11
FP16_K = 12


def _bilinear_taps(lat, Wt, Ht, x, y):
    gh, gw, _ = lat.shape
    gx = (x + 0.5) * gw / Wt - 0.5
    gy = (y + 0.5) * gh / Ht - 0.5
    x0, y0 = np.floor(gx).astype(int), np.floor(gy).astype(int)
    fx, fy = gx - x0, gy - y0
    taps = []
    for dy in (0, 1):
        for dx in (0, 1):
            taps.append((np.clip(y0 + dy, 0, gh - 1), np.clip(x0 + dx, 0, gw - 1),
                         (fx if dx else 1 - fx) * (fy if dy else 1 - fy)))
    return taps


def abs_gradients(p, Wt, Ht, xs, ys, targets):
    """G_abs of every parameter (float64): the gradient of the mean squared
    error with every factor replaced by its absolute value and |e| widened
    by the forward roundings' bound.  A bound for the test, not an expected
    value (those come from the oracle)."""
    p = {k: np.asarray(v, np.float64) for k, v in p.items()}
    n = len(xs)
    t0, t1 = _bilinear_taps(p["lat0"], Wt, Ht, xs, ys), _bilinear_taps(p["lat1"], Wt, Ht, xs, ys)
    F = np.concatenate([sum(w[:, None] * p["lat0"][yi, xi] for yi, xi, w in t0),
                        sum(w[:, None] * p["lat1"][yi, xi] for yi, xi, w in t1)], axis=1)
    H1 = np.maximum(F @ p["w1"].T + p["b1"], 0)
    H2 = np.maximum(H1 @ p["w2"].T + p["b2"], 0)
    Y = H2 @ p["w3"].T + p["b3"]
    Yabs = np.abs(H2) @ np.abs(p["w3"]).T + np.abs(p["b3"])
    E = (np.abs(Y - targets) + 6 * FP16_U * Yabs) * 2.0 / n
    A2 = (E @ np.abs(p["w3"])) * (H2 > 0)
    A1 = (A2 @ np.abs(p["w2"])) * (H1 > 0)
    AF = A1 @ np.abs(p["w1"])
    g = {"w3": E.T @ H2, "b3": E.sum(0), "w2": A2.T @ H1, "b2": A2.sum(0), "w1": A1.T @ np.abs(F),
         "b1": A1.sum(0)}
    for name, taps, sl in (("lat0", t0, slice(0, 8)), ("lat1", t1, slice(8, 16))):
        G = np.zeros(p[name].shape)
        for yi, xi, w in taps:
            np.add.at(G, (yi, xi), np.abs(w)[:, None] * AF[:, sl])
        g[name] = G
    return g


def test_gradients_match_fp64_oracle():
    Wt = Ht = 64
    blocks = synth.random_blocks(Wt, Ht, seed=21)
    tex = _ctf.ctf_texture_create(Wt, Ht, blocks)
    desc = _ctf.train_desc(((16, 16), (8, 8)), batch=1024, total_steps=10)
    tr = _ctf.ctf_trainer_create(tex, desc)
    try:
        g = np.random.default_rng(7)
        params = {"lat0": g.normal(0, 0.7, (16, 16, 8)), "lat1": g.normal(0, 0.7, (8, 8, 8)),
                  "w1": g.normal(0, 0.4, (64, 16)), "b1": g.normal(0, 0.1, 64),
                  "w2": g.normal(0, 0.18, (64, 64)), "b2": g.normal(0, 0.1, 64),
                  "w3": g.normal(0, 0.15, (4, 64)), "b3": g.normal(0.5, 0.1, 4)}
        params = {k: v.astype(np.float32) for k, v in params.items()}
        _ctf.ctf_trainer_set_params(tr, params)
        back = _ctf.ctf_trainer_get_params(tr, desc)
        for k in params:
            np.testing.assert_array_equal(back[k], params[k])
        n = 700  # several CTAs of 128 texels and a ragged tail
        xs, ys = g.integers(0, Wt, n), g.integers(0, Ht, n)
        xy = torch.from_numpy(np.stack([xs, ys], -1).astype(np.int32)).cuda()
        loss, grads = _ctf.ctf_trainer_gradients(tr, desc, xy, n)
        mlp = oracle.MLP((params["lat0"], params["lat1"]), params["w1"], params["b1"], params["w2"],
                         params["b2"], params["w3"], params["b3"], saturate=False)
        ref_loss, ref = oracle.mlp_loss_grad(mlp, Wt, Ht, xs, ys, _decoded(blocks, Wt, Ht, xs, ys))
        dec = _decoded(blocks, Wt, Ht, xs, ys)
        # the loss is summed from FP32 errors of an FP16-operand forward pass
        assert loss == pytest.approx(ref_loss, rel=6 * FP16_U)
        gabs = abs_gradients(params, Wt, Ht, xs, ys, dec)
        for k in _ctf.PARAM_NAMES:
            assert np.abs(ref[k]).max() > 0, k
            err = np.abs(grads[k] - ref[k]).max()
            bound = FP16_K * FP16_U * gabs[k].max() + 1e-9
            assert err <= bound, (k, err, bound)
    finally:
        _ctf.ctf_trainer_destroy(tr)
        _ctf.ctf_texture_destroy(tex)


def _step_texels(seed, step, batch, Wt, Ht):
    """Texels a training step samples: Philox4x32-10 of counter (i, step,
    0x5A4D, 0) under the trainer's seed, scaled to the texture by a 32-bit
    fixed-point multiply."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    r = np.stack([oracle.philox4x32_10((i, step, 0x5A4D, 0), key) for i in range(batch)]).astype(np.uint64)
    return (r[:, 0] * Wt) >> 32, (r[:, 1] * Ht) >> 32


def test_training_steps_follow_adam_on_fp64_gradients():
    """Two ctf_trainer_step calls against Adam (bias-corrected, learning
    rate decaying linearly) applied in FP64 to the gradients the steps used:
    ctf_trainer_gradients on each step's sampled texels (Philox, as the
    step draws them) gives the same sums the step computes (the same
    kernel, the same split of the batch, fixed-point sums).  Elements whose
    gradients are well above the FP32 rounding of the moments must move by
    the reference update within 2e-3 lr; every element stays within Adam's
    step bound.  (The gradients' own accuracy is the gradient test's.)"""
    Wt = Ht = 64
    blocks = synth.random_blocks(Wt, Ht, seed=22)
    tex = _ctf.ctf_texture_create(Wt, Ht, blocks)
    batch, total, seed = 1024, 10, 0x1234_0000_0077
    lr_w, lr_l, frac, b1, b2, eps = 3e-3, 3e-2, 0.1, 0.9, 0.99, 1e-10
    desc = _ctf.train_desc(((16, 16), (8, 8)), batch=batch, total_steps=total, lr_weights=lr_w, lr_latents=lr_l,
                           lr_final_frac=frac, beta1=b1, beta2=b2, eps=eps, seed=seed)
    tr = _ctf.ctf_trainer_create(tex, desc)
    try:
        g = np.random.default_rng(8)
        p0 = {"lat0": g.normal(0, 0.7, (16, 16, 8)), "lat1": g.normal(0, 0.7, (8, 8, 8)),
              "w1": g.normal(0, 0.4, (64, 16)), "b1": g.normal(0, 0.1, 64),
              "w2": g.normal(0, 0.18, (64, 64)), "b2": g.normal(0, 0.1, 64),
              "w3": g.normal(0, 0.15, (4, 64)), "b3": g.normal(0.5, 0.1, 4)}
        p0 = {k: v.astype(np.float32) for k, v in p0.items()}
        _ctf.ctf_trainer_set_params(tr, p0)
        p = {k: v.astype(np.float64) for k, v in p0.items()}
        m = {k: np.zeros_like(v) for k, v in p.items()}
        v2 = {k: np.zeros_like(v) for k, v in p.items()}
        grads, got = [], []
        for st in range(2):
            xs, ys = _step_texels(seed, st, batch, Wt, Ht)
            xy = torch.from_numpy(np.stack([xs, ys], -1).astype(np.int32)).cuda()
            _, gr = _ctf.ctf_trainer_gradients(tr, desc, xy, batch)
            gr = {k: v.astype(np.float64) for k, v in gr.items()}
            grads.append(gr)
            _ctf.ctf_trainer_step(tr, 1)
            _ctf.ctf_sync_check()
            got.append(_ctf.ctf_trainer_get_params(tr, desc))
            sched = 1.0 - (1.0 - frac) * min(1.0, st / total)
            t = st + 1
            for k in p:
                lr = (lr_l if k.startswith("lat") else lr_w) * sched
                m[k] = b1 * m[k] + (1 - b1) * gr[k]
                v2[k] = b2 * v2[k] + (1 - b2) * gr[k] ** 2
                p[k] = p[k] - lr / (1 - b1 ** t) * m[k] / (np.sqrt(v2[k] / (1 - b2 ** t)) + eps)
        for k in p:
            lr = lr_l if k.startswith("lat") else lr_w
            u_ref = p[k] - p0[k]
            u_gpu = got[1][k].astype(np.float64) - p0[k]
            well = np.ones(u_ref.shape, bool)
            for gr in grads:
                well &= np.abs(gr[k]) > 1e-2 * np.abs(gr[k]).max()
            assert well.mean() > 0.3, (k, well.mean())
            err = np.abs(u_gpu - u_ref)[well].max()
            assert err <= 2e-3 * lr, (k, err, lr)
            assert np.abs(u_gpu).max() <= 2.5 * lr, k
    finally:
        _ctf.ctf_trainer_destroy(tr)
        _ctf.ctf_texture_destroy(tex)


@pytest.fixture(scope="module")
def procedural256():
    rgba = synth.procedural_rgba8(256, seed=1)
    blocks = synth.encode_blocks(rgba)
    tex = _ctf.ctf_texture_create(256, 256, blocks)
    yield tex, blocks
    _ctf.ctf_texture_destroy(tex)


def _psnr(mse):
    return -10.0 * math.log10(max(mse, 1e-30))


def test_training_gains_over_the_untrained_network(procedural256):
    """What the trained network gains: PSNR of the learned decode against the
    exact decode before and after training, both quantised to FP16."""
    tex, _ = procedural256
    desc = _ctf.train_desc(((64, 64), (32, 32)), batch=32768, total_steps=300)
    tr = _ctf.ctf_trainer_create(tex, desc)
    try:
        before = _ctf.ctf_trainer_export(tr, _ctf.CTF_EVAL_MLP_FP16)
        mse0, _ = _ctf.ctf_texture_compare(tex, before)
        _ctf.ctf_texture_destroy(before)
        _ctf.ctf_trainer_step(tr, 300)
        after = _ctf.ctf_trainer_export(tr, _ctf.CTF_EVAL_MLP_FP16)
        mse1, mx1 = _ctf.ctf_texture_compare(tex, after)
        _ctf.ctf_sync_check()
        _ctf.ctf_texture_destroy(after)
        print(f"PSNR untrained {_psnr(mse0):.2f} dB -> trained {_psnr(mse1):.2f} dB (max abs {mx1:.3f})")
        assert _psnr(mse1) > _psnr(mse0) + 12.0
        assert _psnr(mse1) > 26.0
        assert _ctf.ctf_trainer_steps_done(tr) == 300
    finally:
        _ctf.ctf_trainer_destroy(tr)


def test_checkpoint_resume_is_bit_identical(procedural256):
    tex, _ = procedural256
    desc = _ctf.train_desc(((64, 64), (32, 32)), batch=8192, total_steps=20, seed=99)
    tr = _ctf.ctf_trainer_create(tex, desc)
    d = tempfile.mkdtemp()
    path = os.path.join(d, "ckpt.bin")
    try:
        _ctf.ctf_trainer_step(tr, 6)
        _ctf.ctf_trainer_save(tr, path)
        _ctf.ctf_trainer_step(tr, 6)
        straight = _ctf.ctf_trainer_get_params(tr, desc)
        tr2 = _ctf.ctf_trainer_load(tex, path)
        try:
            assert _ctf.ctf_trainer_steps_done(tr2) == 6
            _ctf.ctf_trainer_step(tr2, 6)
            resumed = _ctf.ctf_trainer_get_params(tr2, desc)
        finally:
            _ctf.ctf_trainer_destroy(tr2)
        for k in straight:
            assert np.array_equal(straight[k].view(np.uint32), resumed[k].view(np.uint32)), k
        # a corrupted checkpoint is refused
        raw = bytearray(open(path, "rb").read())
        raw[100] ^= 0x40
        bad = os.path.join(d, "bad.bin")
        open(bad, "wb").write(bytes(raw))
        with pytest.raises(_ctf.CtfError) as ei:
            _ctf.ctf_trainer_load(tex, bad)
        assert ei.value.status == _ctf.CTF_ERR_CORRUPT
    finally:
        _ctf.ctf_trainer_destroy(tr)


def test_fp8_export_matches_fp64_oracle(procedural256):
    """E4M3 activations: relative rounding 2^-4 plus half the subnormal
    spacing (2^-10 in scaled units) per input, propagated through |W_eff|
    as for FP16; W_eff = s_o q[o][k] / a_k exactly as stored."""
    tex, _ = procedural256
    desc = _ctf.train_desc(((64, 64), (32, 32)), batch=16384, total_steps=60)
    tr = _ctf.ctf_trainer_create(tex, desc)
    try:
        _ctf.ctf_trainer_step(tr, 60)
        t8 = _ctf.ctf_trainer_export(tr, _ctf.CTF_EVAL_MLP_FP8)
        st = _ctf.ctf_mlp_export(t8, ((64, 64, 8), (32, 32, 8)))
        weff = [st["ws0"][:, None] * st["w1"] / st["as0"][None, :],
                st["ws1"][:, None] * st["w2"] / st["as1"][None, :],
                st["ws2"][:, None] * st["w3"] / st["as2"][None, :]]
        weff = [w.astype(np.float64) for w in weff]
        mlp = oracle.MLP((st["lat0"], st["lat1"]), weff[0], st["b1"], weff[1], st["b2"], weff[2], st["b3"])
        g = np.random.default_rng(3)
        n = 2000
        xs, ys = g.integers(0, 256, n), g.integers(0, 256, n)
        d_xy = torch.from_numpy(np.stack([xs, ys], -1).astype(np.int32)).cuda()
        out = torch.empty((n, 4), device="cuda")
        _ctf.ctf_mlp_decode(t8, d_xy, n, out)
        _ctf.ctf_sync_check()
        got = out.cpu().numpy()
        ref = oracle.mlp_decode(mlp, 256, 256, xs, ys)
        F = np.stack([oracle.mlp_features(mlp, 256, 256, int(x), int(y)) for x, y in zip(xs, ys)])
        h1 = np.maximum(F @ weff[0].T + st["b1"], 0)
        h2 = np.maximum(h1 @ weff[1].T + st["b2"], 0)
        u = 2.0 ** -4
        e_f = u * np.abs(F) + 2.0 ** -10 * st["as0"]
        e_h1 = u * h1 + 2.0 ** -10 * st["as1"] + e_f @ np.abs(weff[0]).T
        e_h2 = u * h2 + 2.0 ** -10 * st["as2"] + e_h1 @ np.abs(weff[1]).T
        tol = 2.0 * (e_h2 @ np.abs(weff[2]).T) + 1e-5
        err = np.abs(got - ref)
        assert np.all(err <= tol), (err.max(), (err / tol).max())
        _ctf.ctf_texture_destroy(t8)
    finally:
        _ctf.ctf_trainer_destroy(tr)


def _params_of(tex, desc, fp8):
    shapes = ((desc.latent_h[0], desc.latent_w[0], 8), (desc.latent_h[1], desc.latent_w[1], 8))
    st = _ctf.ctf_mlp_export(tex, shapes)
    return {k: v for k, v in st.items() if fp8 or not (k.startswith("ws") or k.startswith("as"))}


def test_mlp_train_is_the_trainer_in_one_call(procedural256):
    """ctf_mlp_train gives the texture of create + step + export, bit for
    bit (training is deterministic), and reports its error against the exact
    texture as ctf_texture_compare measures it."""
    tex, _ = procedural256
    desc = _ctf.train_desc(((64, 64), (32, 32)), batch=8192, total_steps=40, seed=5)
    for mode in (_ctf.CTF_EVAL_MLP_FP16, _ctf.CTF_EVAL_MLP_FP8):
        one, rep = _ctf.ctf_mlp_train(tex, desc, mode)
        tr = _ctf.ctf_trainer_create(tex, desc)
        try:
            _ctf.ctf_trainer_step(tr, 40)
            ref = _ctf.ctf_trainer_export(tr, mode)
        finally:
            _ctf.ctf_trainer_destroy(tr)
        try:
            fp8 = mode == _ctf.CTF_EVAL_MLP_FP8
            a, b = _params_of(one, desc, fp8), _params_of(ref, desc, fp8)
            for k in a:
                assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), (mode, k)
            mse, mx = _ctf.ctf_texture_compare(tex, one)
            assert rep["steps"] == 40 and rep["texels"] == 40 * 8192 and rep["seconds"] > 0
            # the mean is summed in parallel, in no fixed order
            assert rep["mse_rgb"] == pytest.approx(mse, rel=1e-12) and rep["max_abs"] == mx
            assert rep["psnr_db"] == pytest.approx(_psnr(mse), abs=1e-9)
        finally:
            _ctf.ctf_texture_destroy(one)
            _ctf.ctf_texture_destroy(ref)
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_mlp_train(tex, desc, _ctf.CTF_EVAL_BLOCK)
    assert ei.value.status == _ctf.CTF_ERR_ARG


def test_texture_checkpoints_round_trip_bit_for_bit(procedural256):
    """A block, an FP16 and an FP8 texture saved and loaded back: the same
    stored parameters, the same decoded texels and the same filtered image
    bit for bit; a flipped byte or a cut file is refused."""
    tex, _ = procedural256
    desc = _ctf.train_desc(((64, 64), (32, 32)), batch=8192, total_steps=30, seed=8)
    tr = _ctf.ctf_trainer_create(tex, desc)
    try:
        _ctf.ctf_trainer_step(tr, 30)
        learned = {m: _ctf.ctf_trainer_export(tr, m) for m in (_ctf.CTF_EVAL_MLP_FP16, _ctf.CTF_EVAL_MLP_FP8)}
    finally:
        _ctf.ctf_trainer_destroy(tr)
    sc = synth.perspective_view(200, 120, 256, 256, 1.0, 8.0, seed=4)
    d_uv, d_jac, d_cov = (torch.from_numpy(a).cuda() for a in (sc.uv, sc.jac, sc.coverage))
    g = np.random.default_rng(2)
    xy = torch.from_numpy(np.stack([g.integers(0, 256, 500), g.integers(0, 256, 500)], -1).astype(np.int32)).cuda()

    def filtered(t):
        out = torch.empty((sc.H, sc.W, 4), device="cuda")
        ev = torch.empty((sc.H, sc.W), dtype=torch.uint8, device="cuda")
        _ctf.ctf_filter(t, d_uv, d_jac, d_cov, sc.W, sc.H, 0, "mask", 3, {"mask_dim": 11}, out, ev)
        _ctf.ctf_sync_check()
        return out.cpu().numpy(), ev.cpu().numpy()

    d = tempfile.mkdtemp()
    try:
        for name, t in (("block", tex), ("fp16", learned[_ctf.CTF_EVAL_MLP_FP16]),
                        ("fp8", learned[_ctf.CTF_EVAL_MLP_FP8])):
            path = os.path.join(d, name + ".ctftex")
            _ctf.ctf_checkpoint_save(t, path)
            back = _ctf.ctf_checkpoint_load(path)
            try:
                a, b = filtered(t), filtered(back)
                assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32)), name
                assert np.array_equal(a[1], b[1]), name
                if name != "block":
                    fp8 = name == "fp8"
                    pa, pb = _params_of(t, desc, fp8), _params_of(back, desc, fp8)
                    for k in pa:
                        assert np.array_equal(pa[k].view(np.uint32), pb[k].view(np.uint32)), (name, k)
                    oa, ob = torch.empty((500, 4), device="cuda"), torch.empty((500, 4), device="cuda")
                    _ctf.ctf_mlp_decode(t, xy, 500, oa)
                    _ctf.ctf_mlp_decode(back, xy, 500, ob)
                    _ctf.ctf_sync_check()
                    assert torch.equal(oa, ob), name
            finally:
                _ctf.ctf_texture_destroy(back)
            raw = bytearray(open(path, "rb").read())
            for bad_raw in (raw[:-1], raw[:60] + bytes([raw[60] ^ 1]) + raw[61:]):
                bad = os.path.join(d, "bad.ctftex")
                open(bad, "wb").write(bytes(bad_raw))
                with pytest.raises(_ctf.CtfError) as ei:
                    _ctf.ctf_checkpoint_load(bad)
                assert ei.value.status == _ctf.CTF_ERR_CORRUPT, name
    finally:
        for t in learned.values():
            _ctf.ctf_texture_destroy(t)


def test_stream_status_is_the_sync_check():
    _ctf.ctf_stream_status()
    _ctf.ctf_selftest_bounded_wait(1 << 10)
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_stream_status()
    assert ei.value.status == _ctf.CTF_ERR_TIMEOUT
    _ctf.ctf_stream_status()
