"""Pins of the FP64 network reference (2D and 3D): convolution against scipy's
correlation, pooling / upsampling against their closed forms, the analytic
backward pass against central finite differences, Adam against its formula."""
import math

import numpy as np
import pytest
import scipy.signal

from oracle import nn


def _params(n, C, seed):
    rng = np.random.default_rng(seed)
    return {k: rng.standard_normal(s) * (0.4 if k.endswith(".w") else 0.1)
            for k, s in nn.param_shapes(n, C)}


@pytest.mark.parametrize("d", [1, 2])
def test_conv_matches_scipy_correlate(d):
    rng = np.random.default_rng(d)
    C, O, H = 3, 2, 11
    inp = rng.standard_normal((C, H, H))
    W = rng.standard_normal((O, C, 3, 3))
    bias = rng.standard_normal(O)
    got = nn.conv_fwd(inp, W, bias, d)
    for o in range(O):
        ref = np.full((H, H), bias[o])
        for c in range(C):
            k = np.zeros((2 * d + 1, 2 * d + 1))
            k[::d, ::d] = W[o, c]
            ref += scipy.signal.correlate2d(inp[c], k, mode="same", boundary="fill")
        assert np.allclose(got[o], ref, atol=1e-12)


def test_pool_and_upsample_closed_forms():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 8, 8))
    p = nn.avgpool2(x)
    assert p.shape == (2, 4, 4)
    assert np.isclose(p.sum() * 4, x.sum())
    assert np.allclose(nn.avgpool2(np.full((1, 7, 7), 3.0)), 3.0)
    # half-pixel bilinear x2: interior out[2i] = .75 in[i] + .25 in[i-1],
    # out[2i+1] = .75 in[i] + .25 in[i+1]; edges clamp.
    z = rng.standard_normal((1, 5, 5))
    u = nn.upsample(z, 10)
    row = z[0, 2]
    col = np.empty(10)
    for i in range(5):
        col[2 * i] = 0.75 * row[i] + 0.25 * row[max(i - 1, 0)]
        col[2 * i + 1] = 0.75 * row[i] + 0.25 * row[min(i + 1, 4)]
    ref_rows = np.empty((5, 10))
    for r in range(5):
        rr = z[0, r]
        for i in range(5):
            ref_rows[r, 2 * i] = 0.75 * rr[i] + 0.25 * rr[max(i - 1, 0)]
            ref_rows[r, 2 * i + 1] = 0.75 * rr[i] + 0.25 * rr[min(i + 1, 4)]
    ref = np.empty((10, 10))
    for c in range(10):
        cc = ref_rows[:, c]
        for i in range(5):
            ref[2 * i, c] = 0.75 * cc[i] + 0.25 * cc[max(i - 1, 0)]
            ref[2 * i + 1, c] = 0.75 * cc[i] + 0.25 * cc[min(i + 1, 4)]
    assert np.allclose(u[0], ref, atol=1e-14)
    assert np.allclose(nn.upsample(np.full((1, 4, 4), 2.0), 13), 2.0)
    # adjointness of the backward maps
    g = rng.standard_normal((1, 10, 10))
    assert np.isclose((u * g).sum(), (z * nn.upsample_bwd(g, 5)).sum())
    g8 = rng.standard_normal((2, 4, 4))
    assert np.isclose((p * g8).sum(), (x * nn.avgpool2_bwd(g8, 8, 8)).sum())


def test_level_sizes():
    assert nn.level_sizes(256) == [256, 128, 64, 32, 16, 8]
    assert nn.level_sizes(32) == [32, 16, 8]
    assert nn.level_sizes(100) == [100, 50, 25, 12]
    assert nn.level_sizes(4) == [4]


def test_gradients_vs_central_differences():
    n, C = 16, 4
    params = _params(n, C, 1)
    rng = np.random.default_rng(2)
    inputs = rng.standard_normal((2, n * n))
    targets = rng.standard_normal((2, n * n))
    _, grads = nn.loss_and_grads(params, inputs, targets, n)
    eps = 1e-6
    for name in params:
        flat = params[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(4, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            lp, _ = nn.loss_and_grads(params, inputs, targets, n)
            flat[i] = old - eps
            lm, _ = nn.loss_and_grads(params, inputs, targets, n)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            an = grads[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3), (name, i, fd, an)


def test_adam_formula():
    theta = np.array([1.0, -2.0, 0.5])
    g1 = np.array([0.3, -0.1, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    th1, m, v = nn.adam_update(theta, m, v, g1, 1, lr=0.01)
    # step 1: mhat = g, vhat = g^2 -> theta - lr g/(|g| + eps)
    assert np.allclose(th1, theta - 0.01 * g1 / (np.abs(g1) + 1e-8), atol=1e-15)
    g2 = np.array([0.1, 0.2, -0.4])
    th2, m2, v2 = nn.adam_update(th1, m, v, g2, 2, lr=0.01)
    mm = 0.9 * 0.1 * g1 + 0.1 * g2
    vv = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    step = 0.01 * (mm / (1 - 0.81)) / (np.sqrt(vv / (1 - 0.999 ** 2)) + 1e-8)
    assert np.allclose(th2, th1 - step, atol=1e-14)


def test_training_reduces_loss():
    """A few full-batch Adam steps on one pair lower the loss (sanity of the
    loss/gradient/update chain as a whole)."""
    n, C = 16, 4
    params = _params(n, C, 5)
    rng = np.random.default_rng(6)
    u = rng.standard_normal((1, n * n))
    t = rng.standard_normal((1, n * n)) * 0.1
    state = {k: (np.zeros_like(p), np.zeros_like(p)) for k, p in params.items()}
    l0, _ = nn.loss_and_grads(params, u, t, n)
    for step in range(1, 31):
        _, g = nn.loss_and_grads(params, u, t, n)
        for k in params:
            params[k], m, v = nn.adam_update(params[k], *state[k], g[k], step, lr=1e-2)
            state[k] = (m, v)
    l1, _ = nn.loss_and_grads(params, u, t, n)
    assert l1 < 0.5 * l0


# ---------------------------------------------------------------- 3D network

def _params3(n, C, seed):
    rng = np.random.default_rng(seed)
    return {k: rng.standard_normal(s) * (0.3 if k.endswith(".w") else 0.1)
            for k, s in nn.param_shapes(n, C, dim=3)}


@pytest.mark.parametrize("d", [1, 2])
def test_conv3d_matches_scipy_correlate(d):
    import scipy.ndimage
    rng = np.random.default_rng(10 + d)
    C, O, H = 2, 2, 7
    inp = rng.standard_normal((C, H, H, H))
    W = rng.standard_normal((O, C, 3, 3, 3))
    bias = rng.standard_normal(O)
    got = nn.conv_fwd(inp, W, bias, d)
    for o in range(O):
        ref = np.full((H, H, H), bias[o])
        for c in range(C):
            k = np.zeros((2 * d + 1,) * 3)
            k[::d, ::d, ::d] = W[o, c]
            ref += scipy.ndimage.correlate(inp[c], k, mode="constant", cval=0.0)
        assert np.allclose(got[o], ref, atol=1e-12)


def test_pool3d_and_trilinear_closed_forms():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 8, 8, 8))
    p = nn.avgpool2(x)
    assert p.shape == (2, 4, 4, 4)
    assert np.isclose(p[1, 2, 1, 3], x[1, 4:6, 2:4, 6:8].mean())
    assert np.allclose(nn.avgpool2(np.full((1, 7, 7, 7), 3.0)), 3.0)
    # trilinear upsampling written out corner by corner at sampled points
    z = rng.standard_normal((1, 5, 5, 5))
    n = 12
    u = nn.upsample(z, n)

    def src(i):
        s = max((i + 0.5) * 5 / n - 0.5, 0.0)
        i0 = min(int(math.floor(s)), 4)
        return i0, min(i0 + 1, 4), s - i0

    for (i, j, k) in [(0, 0, 0), (3, 7, 11), (11, 5, 2), (6, 6, 6)]:
        z0, z1, lz = src(i)
        y0, y1, ly = src(j)
        x0, x1, lx = src(k)
        ref = 0.0
        for zz, wz in ((z0, 1 - lz), (z1, lz)):
            for yy, wy in ((y0, 1 - ly), (y1, ly)):
                for xx, wx in ((x0, 1 - lx), (x1, lx)):
                    ref += wz * wy * wx * z[0, zz, yy, xx]
        assert abs(u[0, i, j, k] - ref) < 1e-13
    assert np.allclose(nn.upsample(np.full((1, 4, 4, 4), 2.0), 9), 2.0)
    g = rng.standard_normal((1, n, n, n))
    assert np.isclose((u * g).sum(), (z * nn.upsample_bwd(g, 5)).sum())
    g4 = rng.standard_normal((2, 4, 4, 4))
    assert np.isclose((p * g4).sum(), (x * nn.avgpool2_bwd(g4, 8, 8, 8)).sum())


def test_3d_gradients_vs_central_differences():
    n, C = 8, 3
    params = _params3(n, C, 7)
    rng = np.random.default_rng(8)
    inputs = rng.standard_normal((1, n ** 3))
    targets = rng.standard_normal((1, n ** 3))
    _, grads = nn.loss_and_grads(params, inputs, targets, n, dim=3)
    eps = 1e-6
    for name in params:
        flat = params[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(3, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            lp, _ = nn.loss_and_grads(params, inputs, targets, n, dim=3)
            flat[i] = old - eps
            lm, _ = nn.loss_and_grads(params, inputs, targets, n, dim=3)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            an = grads[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3), (name, i, fd, an)


def test_grown_network_gradients_and_identity_start():
    """Adaptive growth (Sec. 2.1, residual blocks appended before the output
    layer): with zero weights an extra block is the identity, so the grown
    network computes the same output; gradients of the grown network match
    central differences."""
    n, C = 16, 3
    rng = np.random.default_rng(21)
    base = {k: rng.standard_normal(s) * (0.4 if k.endswith(".w") else 0.1)
            for k, s in nn.param_shapes(n, C)}
    grown = dict(base)
    for k, s in nn.param_shapes(n, C, extra_blocks=2)[len(base):]:
        grown[k] = np.zeros(s)
    u = rng.standard_normal(n * n)
    assert np.allclose(nn.forward(base, u, n), nn.forward(grown, u, n), atol=1e-14)
    for k, s in nn.param_shapes(n, C, extra_blocks=2)[len(base):]:
        grown[k] = rng.standard_normal(s) * (0.3 if k.endswith(".w") else 0.1)
    inputs = rng.standard_normal((1, n * n))
    targets = rng.standard_normal((1, n * n))
    _, grads = nn.loss_and_grads(grown, inputs, targets, n)
    eps = 1e-6
    for name in ("res1.w", "res2.b", "dil.w", "level0.w", "in.w"):
        flat = grown[name].reshape(-1)
        for i in rng.choice(flat.size, size=3, replace=False):
            old = flat[i]
            flat[i] = old + eps
            lp, _ = nn.loss_and_grads(grown, inputs, targets, n)
            flat[i] = old - eps
            lm, _ = nn.loss_and_grads(grown, inputs, targets, n)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            an = grads[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3), (name, i, fd, an)
