"""Pins of the FP64 learned-decode oracle: features against scipy's bilinear
interpolation, the forward pass against numpy matmuls, and the backward pass
against central finite differences of the oracle's own loss."""
import numpy as np
import pytest


def _random_mlp(oracle_lib, g, Wt=32, Ht=16, ch=8, hidden=64, grids=((8, 4), (4, 2))):
    lat = [g.normal(0, 0.5, (gh, gw, ch)) for (gw, gh) in grids]
    w1 = g.normal(0, 0.4, (hidden, 2 * ch))
    b1 = g.normal(0, 0.1, hidden)
    w2 = g.normal(0, 0.2, (hidden, hidden))
    b2 = g.normal(0, 0.1, hidden)
    w3 = g.normal(0, 0.2, (4, hidden))
    b3 = g.normal(0.5, 0.1, 4)
    return lat, (w1, b1, w2, b2, w3, b3)


def test_features_match_scipy(oracle_lib):
    from scipy.ndimage import map_coordinates
    g = np.random.default_rng(1)
    Wt, Ht = 32, 16
    lat, p = _random_mlp(oracle_lib, g, Wt, Ht)
    m = oracle_lib.MLP(lat, *p)
    for x, y in [(0, 0), (31, 15), (5, 7), (17, 2), (30, 1)]:
        f = oracle_lib.mlp_features(m, Wt, Ht, x, y)
        ref = []
        for L in lat:
            gh, gw = L.shape[:2]
            gx = (x + 0.5) * gw / Wt - 0.5
            gy = (y + 0.5) * gh / Ht - 0.5
            for c in range(L.shape[2]):
                ref.append(map_coordinates(L[..., c], [[gy], [gx]], order=1, mode="nearest")[0])
        np.testing.assert_allclose(f, ref, rtol=1e-13, atol=1e-14)


def test_forward_matches_numpy(oracle_lib):
    g = np.random.default_rng(2)
    Wt, Ht = 32, 16
    lat, (w1, b1, w2, b2, w3, b3) = _random_mlp(oracle_lib, g, Wt, Ht)
    m = oracle_lib.MLP(lat, w1, b1, w2, b2, w3, b3, saturate=False)
    ms = oracle_lib.MLP(lat, w1, b1, w2, b2, w3, b3, saturate=True)
    xs = g.integers(0, Wt, 50)
    ys = g.integers(0, Ht, 50)
    F = np.stack([oracle_lib.mlp_features(m, Wt, Ht, int(x), int(y)) for x, y in zip(xs, ys)])
    h1 = np.maximum(F @ w1.T + b1, 0)
    h2 = np.maximum(h1 @ w2.T + b2, 0)
    ref = h2 @ w3.T + b3
    out = oracle_lib.mlp_decode(m, Wt, Ht, xs, ys)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)
    outs = oracle_lib.mlp_decode(ms, Wt, Ht, xs, ys)
    np.testing.assert_allclose(outs, np.clip(ref, 0, 1), rtol=1e-12, atol=1e-12)


def test_backward_matches_finite_differences(oracle_lib):
    g = np.random.default_rng(3)
    Wt, Ht = 32, 16
    lat, params = _random_mlp(oracle_lib, g, Wt, Ht, hidden=16)
    names = ["w1", "b1", "w2", "b2", "w3", "b3"]
    xs = g.integers(0, Wt, 24)
    ys = g.integers(0, Ht, 24)
    tgt = g.uniform(0, 1, (24, 4))

    def loss_of(lat_, params_):
        mm = oracle_lib.MLP(lat_, *params_, saturate=False)
        return oracle_lib.mlp_loss_grad(mm, Wt, Ht, xs, ys, tgt)

    loss, grads = loss_of(lat, params)
    eps = 1e-6
    checked = 0
    for pi, name in enumerate(names):
        arr = params[pi]
        flat_idx = g.choice(arr.size, size=min(6, arr.size), replace=False)
        for fi in flat_idx:
            idx = np.unravel_index(fi, arr.shape)
            plus = [a.copy() for a in params]
            minus = [a.copy() for a in params]
            plus[pi][idx] += eps
            minus[pi][idx] -= eps
            fd = (loss_of(lat, plus)[0] - loss_of(lat, minus)[0]) / (2 * eps)
            an = grads[name][idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, idx, fd, an)
            checked += 1
    for gi, key in enumerate(("lat0", "lat1")):
        L = lat[gi]
        for fi in g.choice(L.size, size=6, replace=False):
            idx = np.unravel_index(fi, L.shape)
            plus = [a.copy() for a in lat]
            minus = [a.copy() for a in lat]
            plus[gi][idx] += eps
            minus[gi][idx] -= eps
            fd = (loss_of(plus, params)[0] - loss_of(minus, params)[0]) / (2 * eps)
            an = grads[key][idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (key, idx, fd, an)
            checked += 1
    assert checked >= 40
    # the loss itself: mean over the batch of the squared error summed over channels
    mm = oracle_lib.MLP(lat, *params, saturate=False)
    y = oracle_lib.mlp_decode(mm, Wt, Ht, xs, ys)
    assert loss == pytest.approx(((y - tgt) ** 2).sum(1).mean(), rel=1e-12)
