"""Learned coarse-grid correction: BF16 tensor-core CNN kernels against the FP64 oracle.

Tolerances: the GPU rounds weights, features and every activation to BF16
(8-bit significand, relative rounding 2^-9) and accumulates in FP32.  Over four
layers that gives about 1e-2 relative error in the output and the gradients
(measured by the relative L2 norm); the bounds below are 3e-2 for the output
and 5e-2 for each layer's weight gradient, with a cosine similarity >= 0.998.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _flat(params):
    out = []
    for w, b in params:
        out.append(w.reshape(-1))
        out.append(b)
    return np.concatenate(out)


def _unflat(flat, layers):
    out, o = [], 0
    for cin, cout in layers:
        nw = cout * cin * 9
        out.append((flat[o:o + nw].reshape(cout, cin, 3, 3), flat[o + nw:o + nw + cout]))
        o += nw + cout
    return out


def _state(inputs, nx, ny, seed=3):
    b0, g, ph = inputs.ot_family_params(seed, 1)
    w = inputs.orszag_tang(nx, ny, b0=b0, gamma=g, phases=ph, noise=1e-2, seed=seed)
    return w.astype(np.float32).astype(np.float64), g


SCALES = np.array([0.25, 0.25, 0.25, 0.5, 0.3, 0.3, 0.15, 10.0])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def setup(inputs_mod):
    from oracle import cnn as ocnn
    nx, ny = 40, 24
    w, g = _state(inputs_mod, nx, ny)
    params = ocnn.init_params(11, last_scale=1.0)
    rng = np.random.default_rng(12)
    params = [(pw, 0.05 * rng.standard_normal(pb.shape)) for pw, pb in params]
    flat = _flat(params).astype(np.float32)
    params64 = _unflat(flat.astype(np.float64), ocnn.LAYERS)
    target = rng.standard_normal((6, ny, nx)).astype(np.float32)
    return nx, ny, w, g, flat, params64, target


def test_forward_matches_oracle(setup):
    import torch
    from oracle import cnn as ocnn
    from paper_1710_06423_b300.sac import CNN
    nx, ny, w, g, flat, params64, _ = setup
    net = CNN(nx, ny)
    net.set_params(flat)
    net.set_scales(SCALES, np.ones(6))
    wd = torch.from_numpy(w.astype(np.float32)).cuda().contiguous()
    pred = torch.zeros((ny * nx, 8), dtype=torch.float32, device="cuda")
    net.forward(wd, g, 1.0 / nx, 1.0 / ny, pred)
    torch.cuda.synchronize()
    got = pred.cpu().numpy()[:, :6].T.reshape(6, ny, nx)
    x = ocnn.features(w, g, 1.0 / nx, 1.0 / ny, SCALES)
    ref, _ = ocnn.forward(params64, x)
    assert _rel(got, ref) <= 3e-2, _rel(got, ref)
    net.close()


def test_gradients_match_oracle(setup):
    import torch
    from oracle import cnn as ocnn
    from paper_1710_06423_b300.sac import CNN
    nx, ny, w, g, flat, params64, target = setup
    net = CNN(nx, ny)
    net.set_params(flat)
    net.set_scales(SCALES, np.ones(6))
    wd = torch.from_numpy(w.astype(np.float32)).cuda().contiguous()
    # out_scale = 1: the target (next - w) equals `target` up to FP32 rounding
    nd = torch.from_numpy((w.astype(np.float32) + target).astype(np.float32)).cuda().contiguous()
    target = (nd.cpu().numpy().astype(np.float64) - w.astype(np.float32).astype(np.float64)).astype(np.float32)
    loss, grads = net.grads(wd, nd, g, 1.0 / nx, 1.0 / ny)
    x = ocnn.features(w, g, 1.0 / nx, 1.0 / ny, SCALES)
    ref_loss, ref_grads = ocnn.loss_and_grads(params64, x, target.astype(np.float64))
    assert abs(loss - ref_loss) <= 3e-2 * ref_loss
    gg = _unflat(grads.astype(np.float64), ocnn.LAYERS)
    for k in range(4):
        for a, b in ((gg[k][0], ref_grads[k][0]), (gg[k][1], ref_grads[k][1])):
            cos = float(np.sum(a * b) / (np.linalg.norm(a) * np.linalg.norm(b)))
            assert _rel(a, b) <= 5e-2 and cos >= 0.998, (k, _rel(a, b), cos)
    net.close()


def test_training_reduces_loss(setup):
    import torch
    from paper_1710_06423_b300.sac import CNN
    nx, ny, w, g, flat, _, target = setup
    net = CNN(nx, ny)
    net.set_params(flat)
    net.set_scales(SCALES, np.ones(6))
    wd = torch.from_numpy(w.astype(np.float32)).cuda().contiguous()
    # a learnable target: a smooth function of the state itself
    t = 0.1 * w / np.abs(w).max(axis=(1, 2), keepdims=True)
    nd = torch.from_numpy((w + t).astype(np.float32)).cuda().contiguous()
    l0 = net.train_step(wd, nd, g, 1.0 / nx, 1.0 / ny, 2e-3)
    for _ in range(60):
        l = net.train_step(wd, nd, g, 1.0 / nx, 1.0 / ny, 2e-3)
    assert l < 0.3 * l0, (l0, l)
    net.close()


def test_block_average_kernel():
    import torch
    from paper_1710_06423_b300.sac import block_average
    rng = np.random.default_rng(4)
    a = rng.standard_normal((6, 32, 48)).astype(np.float32)
    fine = torch.from_numpy(a).cuda().contiguous()
    out = torch.zeros((6, 8, 12), dtype=torch.float32, device="cuda")
    block_average(fine, 6, 48, 32, 4, out)
    torch.cuda.synchronize()
    ref = a.astype(np.float64).reshape(6, 8, 4, 12, 4).mean(axis=(2, 4))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-6)


def test_apply_adds_scaled_output(setup, inputs_mod):
    import torch
    from paper_1710_06423_b300.sac import CNN, FP32, Solver
    nx, ny, w, g, flat, _, _ = setup
    net = CNN(nx, ny)
    net.set_params(flat)
    osc = np.array([1e-3, 2e-3, 2e-3, 1e-3, 5e-4, 5e-4])
    net.set_scales(SCALES, osc)
    wd = torch.from_numpy(w.astype(np.float32)).cuda().contiguous()
    pred = torch.zeros((ny * nx, 8), dtype=torch.float32, device="cuda")
    net.forward(wd, g, 1.0 / nx, 1.0 / ny, pred)
    torch.cuda.synchronize()
    p = pred.cpu().numpy()[:, :6].T.reshape(6, ny, nx).astype(np.float64)
    with Solver(nx=nx, ny=ny, precision=FP32, gamma=g) as s:
        s.set_state(w, None, 0.0)
        net.apply(s)
        got, t = s.get_state()
        cx, cy = s.cmax()
    pc = p - p.mean(axis=(1, 2), keepdims=True)          # the correction is made conservative
    expect = (w.astype(np.float32) + (osc[:, None, None] * pc).astype(np.float32)).astype(np.float64)
    assert t == 0.0
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-6)
    assert cx > 0 and cy > 0
    net.close()
