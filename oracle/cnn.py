"""FP64 CPU oracle of the learned coarse-grid correction (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.  It shares no code with the CUDA library.

The learned part is not in the paper: it is the "learned coarse-grid
correction" form of the MHD step this repository builds (a small
convolutional network, trained on block-averaged fine-grid snapshots, whose
output is added to the coarse state after each RK4 step).  Every operation is
written from its plain definition with numpy (``np.roll`` for the periodic
shifts, ``np.einsum``/``np.tensordot`` for the channel sums):

  * features (8 channels): the six conserved fields, the kinetic pressure
    p_k = (gamma-1)(e - |m|^2/(2 rho) - |B|^2/2) (section 2 of the paper) and
    the current j_z = D_x B_y - D_y B_x with the section 2 fourth-order central
    difference, each divided by a fixed per-channel scale;
  * conv3x3 with periodic padding:
        y[o, i, j] = b[o] + sum_{c, a, e} W[o, c, a, e] x[c, i + a - 1, j + e - 1]
    (indices mod H, W), a in {0,1,2} the row offset, e the column offset;
  * the network: conv(8->32) ReLU conv(32->32) ReLU conv(32->32) ReLU conv(32->6);
  * the correction u <- u + scale_out * f(features(u));
  * the loss 0.5 * mean over (channel, pixel) of (f(x) - target)^2 and its
    gradient by the chain rule (adjoint of each conv: correlation with the
    flipped kernel for the input, outer products summed over pixels for W);
  * the same network with BF16 storage (``forward_bf16``,
    ``loss_and_grads_bf16``): the form fixes BF16 weights and activations
    with wider accumulation, so these round every stored value to BF16 and
    keep every sum in FP64.
"""
from __future__ import annotations

import numpy as np

LAYERS = ((8, 32), (32, 32), (32, 32), (32, 6))
NFEAT = 8


def conv3x3(x, w, b):
    """Periodic 3x3 convolution (cross-correlation): x [C,H,W], w [O,C,3,3], b [O]."""
    out = np.zeros((w.shape[0],) + x.shape[1:], dtype=np.float64)
    for a in range(3):
        for e in range(3):
            xs = np.roll(x, shift=(1 - a, 1 - e), axis=(1, 2))   # xs[c,i,j] = x[c,i+a-1,j+e-1]
            out += np.tensordot(w[:, :, a, e], xs, axes=([1], [0]))
    return out + b[:, None, None]


def conv3x3_backward(x, w, dy):
    """Gradients of conv3x3 w.r.t. its input, weights and bias given dL/dy."""
    dx = np.zeros_like(x, dtype=np.float64)
    dw = np.zeros_like(w, dtype=np.float64)
    for a in range(3):
        for e in range(3):
            xs = np.roll(x, shift=(1 - a, 1 - e), axis=(1, 2))
            dw[:, :, a, e] = np.tensordot(dy, xs, axes=([1, 2], [1, 2]))
            # y[o,i,j] gets w[o,c,a,e] x[c,i+a-1,j+e-1]  =>  dx[c,k,l] += w[o,c,a,e] dy[o,k-a+1,l-e+1]
            g = np.tensordot(w[:, :, a, e], dy, axes=([0], [0]))     # [C,H,W] at (i,j)
            dx += np.roll(g, shift=(a - 1, e - 1), axis=(1, 2))
    db = dy.sum(axis=(1, 2))
    return dx, dw, db


def forward(params, x):
    """Network output and the per-layer activations needed by backward."""
    acts = [x]
    h = x
    for k, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        if k < len(params) - 1:
            h = np.maximum(z, 0.0)
        else:
            h = z
        acts.append(h)
    return h, acts


def loss_and_grads(params, x, target):
    """0.5 * mean((f(x) - target)^2) and its gradient for every (W, b)."""
    y, acts = forward(params, x)
    r = y - target
    n = r.size
    loss = 0.5 * float(np.sum(r * r)) / n
    dy = r / n
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        w, b = params[k]
        dx, dw, db = conv3x3_backward(acts[k], w, dy)
        grads[k] = (dw, db)
        if k > 0:
            dy = dx * (acts[k] > 0.0)           # ReLU of the layer below
    return loss, grads


def round_bf16(x):
    """Round FP64 values to the nearest BF16 value (8 significant bits, ties to
    even), returned as FP64.  x = m 2^e with m in [0.5, 1): the BF16 neighbours
    are multiples of 2^(e-8), and dividing by that power of two is exact, so
    np.rint (half to even) on the quotient is the rounding itself.  The
    network stores weights and activations in BF16 (finite, normal range)."""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)
    q = np.ldexp(1.0, e - 8)
    return np.rint(x / q) * q


def forward_bf16(params, x):
    """The network with BF16 storage: weights, input features and the three
    hidden activations rounded to BF16; sums, biases and the output in FP64."""
    pb = [(round_bf16(w), b) for w, b in params]
    acts = [round_bf16(x)]
    h = acts[0]
    for k, (w, b) in enumerate(pb):
        z = conv3x3(h, w, b)
        h = round_bf16(np.maximum(z, 0.0)) if k < len(pb) - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grads_bf16(params, x, target, return_stored=False):
    """loss_and_grads with BF16 storage of what the network stores: the output
    gradient r / n and every hidden input gradient are rounded to BF16 after
    the ReLU mask; the weight and bias gradients are exact FP64 sums of those
    stored values.  return_stored: also return (acts, dys), the stored layer
    inputs and the stored output gradient of every layer."""
    pb = [(round_bf16(w), b) for w, b in params]
    y, acts = forward_bf16(params, x)
    r = y - target
    n = r.size
    loss = 0.5 * float(np.sum(r * r)) / n
    dy = round_bf16(r / n)
    grads = [None] * len(pb)
    dys = [None] * len(pb)
    for k in range(len(pb) - 1, -1, -1):
        w, b = pb[k]
        dys[k] = dy
        dx, dw, db = conv3x3_backward(acts[k], w, dy)
        grads[k] = (dw, db)
        if k > 0:
            dy = round_bf16(dx * (acts[k] > 0.0))
    if return_stored:
        return loss, grads, (acts, dys)
    return loss, grads


def dcen_periodic(f, axis, h):
    """Section 2 fourth-order central difference with periodic wrap."""
    return (8.0 * (np.roll(f, -1, axis) - np.roll(f, 1, axis)) - (np.roll(f, -2, axis) - np.roll(f, 2, axis))) / (12.0 * h)


def features(w, gamma, dx, dy, scales):
    """8 normalised input channels from a conserved state w [6, ny, nx] (periodic)."""
    rho, mx, my, e, bx, by = w
    pk = (gamma - 1.0) * (e - 0.5 * (mx * mx + my * my) / rho - 0.5 * (bx * bx + by * by))
    jz = dcen_periodic(by, 1, dx) - dcen_periodic(bx, 0, dy)
    f = np.stack([rho, mx, my, e, bx, by, pk, jz])
    return f / np.asarray(scales, dtype=np.float64)[:, None, None]


def init_params(seed, layers=LAYERS, last_scale=0.0):
    """He-uniform weights (zero bias); the last layer scaled by last_scale (0: identity start)."""
    rng = np.random.default_rng(seed)
    out = []
    for k, (cin, cout) in enumerate(layers):
        lim = np.sqrt(6.0 / (9 * cin))
        w = rng.uniform(-lim, lim, (cout, cin, 3, 3))
        if k == len(layers) - 1:
            w = w * last_scale
        out.append((w, np.zeros(cout)))
    return out


def block_average(w, f):
    """Average f x f blocks: [C, H, W] -> [C, H/f, W/f]."""
    c, h, wd = w.shape
    return w.reshape(c, h // f, f, wd // f, f).mean(axis=(2, 4))
