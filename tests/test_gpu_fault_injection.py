"""Host-side fault injection: device allocations that fail.

Every device allocation of the library goes through one routine, and a test
hook (ctf_debug_fail_allocations) makes chosen ones fail as if the GPU were out
of memory, without calling CUDA.  Each entry point that allocates must then
return CTF_ERR_OOM, give back what it had already taken (the library's count
of live allocations comes back to where it was), and leave the context usable:
the next call with the hook disarmed succeeds and gives the same results as a
call that never saw a failure.  No GPU fault is involved; the failure is made
on the host."""
import numpy as np
import pytest

from paper_2506_17770_gb300 import _ctf, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_17770_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield
    _ctf.ctf_debug_fail_allocations(0)


def _learned(seed, Wt, Ht):
    g = np.random.default_rng(seed)
    lat = [g.normal(0, 1.0, (Ht // 4, Wt // 4, 8)).astype(np.float32),
           g.normal(0, 1.0, (Ht // 8, Wt // 8, 8)).astype(np.float32)]
    return lat, (g.normal(0, 0.35, (64, 16)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
                 g.normal(0, 0.18, (64, 64)).astype(np.float32), g.normal(0, 0.1, 64).astype(np.float32),
                 g.normal(0, 0.04, (4, 64)).astype(np.float32), np.array([0.5, 0.5, 0.5, 0.9], np.float32))


def _filter(tex, sc, alg="mask"):
    out = torch.empty((sc.H, sc.W, 4), device="cuda")
    ev = torch.empty((sc.H, sc.W), dtype=torch.uint8, device="cuda")
    st = _ctf.ctf_filter(tex, torch.from_numpy(sc.uv).cuda(), torch.from_numpy(sc.jac).cuda(), None, sc.W, sc.H, 0,
                         alg, 7, None, out, ev, stats=True)
    _ctf.ctf_sync_check()
    return out.cpu().numpy(), ev.cpu().numpy(), st


def _count_allocations(fn):
    """Run fn with the hook disarmed; return its result and how many device
    allocations it attempted."""
    c0 = _ctf.ctf_debug_device_allocations()
    r = fn()
    return r, _ctf.ctf_debug_device_allocations() - c0


def _expect_oom(fn, skip):
    """Fail the allocation after the first `skip` ones; fn must report
    CTF_ERR_OOM and hold nothing afterwards."""
    torch.cuda.synchronize()
    live0 = _ctf.ctf_debug_live_allocations()
    _ctf.ctf_debug_fail_allocations(1, skip=skip)
    try:
        with pytest.raises(_ctf.CtfError) as ei:
            fn()
    finally:
        _ctf.ctf_debug_fail_allocations(0)
    assert ei.value.status == _ctf.CTF_ERR_OOM, str(ei.value)
    assert _ctf.ctf_debug_live_allocations() == live0, "a failed call kept device memory"
    _ctf.ctf_sync_check()  # the context is usable and no error is pending


def test_hook_arguments_are_checked():
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_debug_fail_allocations(-1)
    assert ei.value.status == _ctf.CTF_ERR_ARG
    with pytest.raises(_ctf.CtfError) as ei:
        _ctf.ctf_debug_fail_allocations(1, skip=-2)
    assert ei.value.status == _ctf.CTF_ERR_ARG


def test_block_texture_creation():
    Wt = Ht = 256
    blocks = synth.random_blocks(Wt, Ht)
    sc = synth.magnified_plane(64, 64, Wt, Ht, scale=0.25)
    tex, n = _count_allocations(lambda: _ctf.ctf_texture_create(Wt, Ht, blocks))
    ref = _filter(tex, sc)
    _ctf.ctf_texture_destroy(tex)
    assert n >= 1
    for skip in range(n):
        _expect_oom(lambda: _ctf.ctf_texture_create(Wt, Ht, blocks), skip)
    tex = _ctf.ctf_texture_create(Wt, Ht, blocks)
    try:
        out, ev, st = _filter(tex, sc)
        assert st == ref[2] and st["tiles_success"] > 0
        np.testing.assert_array_equal(ev, ref[1])
        np.testing.assert_array_equal(out.view(np.uint32), ref[0].view(np.uint32))
    finally:
        _ctf.ctf_texture_destroy(tex)


@pytest.mark.parametrize("mode", [_ctf.CTF_EVAL_MLP_FP16, _ctf.CTF_EVAL_MLP_FP8])
def test_learned_texture_creation(mode):
    """Two latent grids and the operand image: failing the first, second or
    third allocation must free the ones before it."""
    Wt = Ht = 64
    lat, p = _learned(3, Wt, Ht)
    kw = {}
    if mode == _ctf.CTF_EVAL_MLP_FP8:
        kw["act_absmax"] = (np.full(16, 4.0, np.float32), np.full(64, 8.0, np.float32), np.full(64, 8.0, np.float32))
    sc = synth.magnified_plane(64, 64, Wt, Ht, scale=0.25)

    def make():
        return _ctf.ctf_texture_create_mlp(Wt, Ht, mode, lat, *p, **kw)

    tex, n = _count_allocations(make)
    ref = _filter(tex, sc)
    _ctf.ctf_texture_destroy(tex)
    assert n == 3
    for skip in range(n):
        _expect_oom(make, skip)
    tex = make()
    try:
        out, ev, st = _filter(tex, sc)
        assert st == ref[2]
        np.testing.assert_array_equal(ev, ref[1])
        np.testing.assert_array_equal(out.view(np.uint32), ref[0].view(np.uint32))
    finally:
        _ctf.ctf_texture_destroy(tex)


def test_trainer_creation_and_one_call_training():
    Wt = Ht = 64
    blocks = synth.random_blocks(Wt, Ht, seed=21)
    tex = _ctf.ctf_texture_create(Wt, Ht, blocks)
    desc = _ctf.train_desc(((16, 16), (8, 8)), batch=512, total_steps=3)
    try:
        tr, n = _count_allocations(lambda: _ctf.ctf_trainer_create(tex, desc))
        _ctf.ctf_trainer_step(tr, 3)
        ref = _ctf.ctf_trainer_get_params(tr, desc)
        _ctf.ctf_trainer_destroy(tr)
        assert n >= 6
        for skip in range(n):
            _expect_oom(lambda: _ctf.ctf_trainer_create(tex, desc), skip)
        tr = _ctf.ctf_trainer_create(tex, desc)
        try:
            _ctf.ctf_trainer_step(tr, 3)
            got = _ctf.ctf_trainer_get_params(tr, desc)
            for k in ref:
                np.testing.assert_array_equal(got[k], ref[k])
        finally:
            _ctf.ctf_trainer_destroy(tr)
        # one-call training: trainer, exported texture, comparison buffers
        res, n = _count_allocations(lambda: _ctf.ctf_mlp_train(tex, desc, _ctf.CTF_EVAL_MLP_FP16))
        _ctf.ctf_texture_destroy(res[0])
        assert n > 6
        for skip in range(0, n, 2):
            _expect_oom(lambda: _ctf.ctf_mlp_train(tex, desc, _ctf.CTF_EVAL_MLP_FP16), skip)
        res2 = _ctf.ctf_mlp_train(tex, desc, _ctf.CTF_EVAL_MLP_FP16)
        _ctf.ctf_texture_destroy(res2[0])
        # same trained texture: the texel error matches (the squared-error
        # sum is accumulated with atomics, so only to rounding)
        for k in ("steps", "texels", "max_abs"):
            assert res2[1][k] == res[1][k], k
        assert res2[1]["mse_rgb"] == pytest.approx(res[1]["mse_rgb"], rel=1e-12)
    finally:
        _ctf.ctf_texture_destroy(tex)


def test_batch_graph_creation():
    Wt = Ht = 128
    blocks = synth.random_blocks(Wt, Ht, seed=5)
    tex = _ctf.ctf_texture_create(Wt, Ht, blocks)
    try:
        views = []
        for i, (W, H) in enumerate(((40, 24), (17, 9), (64, 32))):
            sc = synth.perspective_view(W, H, Wt, Ht, 1.0, 6.0, seed=11, view=i)
            views.append({"tex": tex, "width": W, "height": H, "view_id": i,
                          "uv": torch.from_numpy(sc.uv).cuda(), "jac": torch.from_numpy(sc.jac).cuda(),
                          "coverage": torch.from_numpy(sc.coverage).cuda(),
                          "out_rgba": torch.full((H, W, 4), -1.0, device="cuda"),
                          "out_evals": torch.full((H, W), 9, dtype=torch.uint8, device="cuda")})
        o = _ctf.batch_opts(mask_dim=11)
        _expect_oom(lambda: _ctf.ctf_batch_graph_create(views, "mask", 3, o), 0)
        g = _ctf.ctf_batch_graph_create(views, "mask", 3, o)
        try:
            _ctf.ctf_batch_graph_launch(g)
            _ctf.ctf_sync_check()
        finally:
            _ctf.ctf_batch_graph_destroy(g)
        for v in views:
            out = torch.empty_like(v["out_rgba"])
            ev = torch.empty_like(v["out_evals"])
            _ctf.ctf_filter(tex, v["uv"], v["jac"], v["coverage"], v["width"], v["height"], v["view_id"], "mask",
                            3, {"mask_dim": 11}, out, ev)
            torch.cuda.synchronize()
            assert torch.equal(ev, v["out_evals"])
            assert torch.equal(out.view(torch.int32), v["out_rgba"].view(torch.int32))
    finally:
        _ctf.ctf_texture_destroy(tex)
