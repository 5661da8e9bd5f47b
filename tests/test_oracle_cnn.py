"""Pins of the FP64 CNN oracle (no GPU)."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def cnn():
    from oracle import cnn as c
    return c


def test_conv_equals_fft_cross_correlation(cnn):
    """Periodic 3x3 conv == circular cross-correlation computed through the FFT."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 10, 7))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, w, b)
    H, W = x.shape[1:]
    ref = np.zeros_like(y)
    X = np.fft.fft2(x)
    for o in range(4):
        acc = np.zeros((H, W), dtype=complex)
        for c in range(3):
            k = np.zeros((H, W))
            for a in range(3):
                for e in range(3):
                    # y[i,j] = sum k[a,e] x[i+a-1, j+e-1]: correlation = convolution with the flipped kernel
                    k[(1 - a) % H, (1 - e) % W] += w[o, c, a, e]
            acc += X[c] * np.fft.fft2(k)
        ref[o] = np.real(np.fft.ifft2(acc)) + b[o]
    np.testing.assert_allclose(y, ref, atol=1e-12)


def test_conv_delta_kernel_is_shift(cnn):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 6, 5))
    for a in range(3):
        for e in range(3):
            w = np.zeros((2, 2, 3, 3))
            w[0, 0, a, e] = 1.0
            w[1, 1, a, e] = 1.0
            y = cnn.conv3x3(x, w, np.zeros(2))
            for i in range(6):
                for j in range(5):
                    assert y[0, i, j] == x[0, (i + a - 1) % 6, (j + e - 1) % 5]


def test_conv_adjoint_dot_product(cnn):
    """<conv(x), g> = <x, dx(g)> and <conv_w(x), g> linear in w: dW from the same identity."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((5, 8, 9))
    w = rng.standard_normal((3, 5, 3, 3))
    g = rng.standard_normal((3, 8, 9))
    y = cnn.conv3x3(x, w, np.zeros(3))
    dx, dw, db = cnn.conv3x3_backward(x, w, g)
    assert abs(np.sum(y * g) - np.sum(x * dx)) < 1e-10 * abs(np.sum(y * g))
    assert abs(np.sum(y * g) - np.sum(w * dw)) < 1e-10 * abs(np.sum(y * g))
    np.testing.assert_allclose(db, g.sum(axis=(1, 2)))


def test_loss_gradient_finite_differences(cnn):
    """Backward of the whole 4-layer network against central differences (FP64, rel 1e-6)."""
    rng = np.random.default_rng(3)
    params = cnn.init_params(4, last_scale=0.5)
    x = rng.standard_normal((8, 8, 8))
    t = rng.standard_normal((6, 8, 8))
    loss, grads = cnn.loss_and_grads(params, x, t)
    h = 1e-6
    for k in range(4):
        w, b = params[k]
        for idx in [(0, 0, 1, 1), (w.shape[0] - 1, w.shape[1] - 1, 2, 0), (1, 2, 0, 2)]:
            wp = w.copy(); wp[idx] += h
            wm = w.copy(); wm[idx] -= h
            pp = [(wp if kk == k else ww, bb) for kk, (ww, bb) in enumerate(params)]
            pm = [(wm if kk == k else ww, bb) for kk, (ww, bb) in enumerate(params)]
            fd = (cnn.loss_and_grads(pp, x, t)[0] - cnn.loss_and_grads(pm, x, t)[0]) / (2 * h)
            an = grads[k][0][idx]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)), (k, idx, fd, an)
        bp = b.copy(); bp[0] += h
        bm = b.copy(); bm[0] -= h
        pp = [(ww, bp if kk == k else bb) for kk, (ww, bb) in enumerate(params)]
        pm = [(ww, bm if kk == k else bb) for kk, (ww, bb) in enumerate(params)]
        fd = (cnn.loss_and_grads(pp, x, t)[0] - cnn.loss_and_grads(pm, x, t)[0]) / (2 * h)
        assert abs(fd - grads[k][1][0]) <= 1e-6 * max(1e-3, abs(grads[k][1][0]))


def test_features_closed_forms(cnn):
    """p_k of a uniform state, and j_z of Fourier modes: the fourth-order difference of
    sin(kx) is (8 sin kh - sin 2kh)/(6h) cos(kx)."""
    n = 16
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    rho, vx, vy, p, g = 0.8, 0.3, -0.2, 1.1, 5 / 3
    bx = -0.5 * np.sin(2 * math.pi * Y)
    by = 0.7 * np.sin(4 * math.pi * X)
    e = p / (g - 1) + 0.5 * rho * (vx * vx + vy * vy) + 0.5 * (bx * bx + by * by)
    w = np.stack([rho * np.ones_like(X), rho * vx * np.ones_like(X), rho * vy * np.ones_like(X), e, bx, by])
    f = cnn.features(w, g, h, h, np.ones(8))
    np.testing.assert_allclose(f[6], p, rtol=1e-12)
    k1, k2 = 4 * math.pi, 2 * math.pi
    dby = 0.7 * (8 * math.sin(k1 * h) - math.sin(2 * k1 * h)) / (6 * h) * np.cos(k1 * X)
    dbx = -0.5 * (8 * math.sin(k2 * h) - math.sin(2 * k2 * h)) / (6 * h) * np.cos(k2 * Y)
    np.testing.assert_allclose(f[7], dby - dbx, atol=1e-10)


def test_block_average(cnn):
    a = np.arange(2 * 8 * 8, dtype=float).reshape(2, 8, 8)
    m = cnn.block_average(a, 4)
    assert m.shape == (2, 2, 2)
    assert m[1, 1, 0] == a[1, 4:8, 0:4].mean()


def test_round_bf16_matches_torch_on_fp32_values(cnn):
    """FP32 values (which convert to BF16 without double rounding) round as
    torch's float32 -> bfloat16 conversion does (round to nearest even)."""
    import torch
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.round_bf16(x.astype(np.float64)), ref)


def test_round_bf16_ties_to_even_and_fixed_points(cnn):
    t = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 3 * 2.0 ** -9 * 257 / 256])
    got = cnn.round_bf16(t)
    assert got[0] == 1.0 and got[1] == 1 + 2.0 ** -6 and got[2] == -1.0
    # values with at most 8 significant bits are fixed points, zero included
    v = np.array([0.0, 1.0, -0.75, 255.0, 2.0 ** -40 * 129, -(2.0 ** 30) * 255])
    np.testing.assert_array_equal(cnn.round_bf16(v), v)


def test_bf16_network_is_the_network_when_every_stored_value_is_exact(cnn):
    """With small-integer weights and inputs every stored value (weights,
    activations, r / n and the input gradients) is exactly a BF16 number, so the
    BF16-storage network must equal the FP64 network bit for bit: a pin that
    forward_bf16 / loss_and_grads_bf16 change nothing but the rounding."""
    rng = np.random.default_rng(6)
    layers = ((2, 3), (3, 3), (3, 2))
    params = [(rng.integers(-1, 2, (co, ci, 3, 3)).astype(np.float64), rng.integers(-2, 3, co).astype(np.float64))
              for ci, co in layers]
    x = rng.integers(-2, 3, (2, 4, 4)).astype(np.float64)
    y, acts = cnn.forward(params, x)
    yb, actsb = cnn.forward_bf16(params, x)
    assert np.array_equal(y, yb) and all(np.array_equal(a, b) for a, b in zip(acts, actsb))
    n = y.size                                  # 2 * 4 * 4 = 32: r / n exact for integer r
    target = y - rng.integers(-3, 4, y.shape)
    l0, g0 = cnn.loss_and_grads(params, x, target)
    l1, g1 = cnn.loss_and_grads_bf16(params, x, target)
    assert n == 32 and l0 == l1
    for (a, b), (c, d) in zip(g0, g1):
        assert np.array_equal(a, c) and np.array_equal(b, d)
