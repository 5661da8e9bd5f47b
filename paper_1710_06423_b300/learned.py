"""Learned coarse-grid correction: data from the fine solver, training, evaluation.

A coarse FP32 run (grid n) takes classical RK4 steps of a fixed size dt_c;
after each step the network of ``sac_cnn_*`` adds its correction
u <- u + out_scale * f(features(u)).  The network is trained on pairs the fine
solver generates: the fine run (grid r*n, step dt_c/r) is block-averaged
(r x r) to the coarse grid at times t_k and t_k + dt_c; the coarse solver
steps the first average once, and the target is the remaining difference to
the second, divided by out_scale.  The plain fine solver is both the source of
the training data and the judge of the error (relative L1 per field against
its block average at the horizon).

Every array operation runs in the library's CUDA kernels (solver steps, block
averages, network forward/backward/update, correction); this module only
sequences the calls and keeps device tensors (torch is used for device memory).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs
from .sac import CNN, FP32, Solver, block_average

#: fixed feature scales: rho, m_x, m_y, e, B_x, B_y, p_k, j_z (Orszag-Tang magnitudes)
FEATURE_SCALES = np.array([0.25, 0.25, 0.25, 0.5, 0.3, 0.3, 0.15, 10.0], dtype=np.float32)
LAYERS = ((8, 32), (32, 32), (32, 32), (32, 6))


def init_params(seed: int, last_scale: float = 0.1) -> np.ndarray:
    """He-uniform weights, zero biases, last layer scaled down (flat FP32 layout of sac_cnn)."""
    rng = np.random.default_rng(seed)
    out = []
    for k, (cin, cout) in enumerate(LAYERS):
        lim = math.sqrt(6.0 / (9 * cin))
        w = rng.uniform(-lim, lim, (cout, cin, 3, 3))
        if k == len(LAYERS) - 1:
            w *= last_scale
        out += [w.reshape(-1), np.zeros(cout)]
    return np.concatenate(out).astype(np.float32)


def _dev(w, torch):
    return torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda().contiguous()


def family_state(seed: int, k: int, n: int):
    b0, gamma, phases = inputs.ot_family_params(seed, k)
    return inputs.orszag_tang(n, b0=b0, gamma=gamma, phases=phases), gamma


class Pairs:
    """Training pairs on the device: inputs x' (coarse state after one coarse step)
    and raw residuals r = avg(fine(t + dt_c)) - x'."""

    def __init__(self):
        self.x, self.r, self.gamma = [], [], []

    def __len__(self):
        return len(self.x)


def generate_pairs(pairs: Pairs, seed: int, k: int, n_coarse: int, ratio: int, dt_c: float, n_steps: int,
                   every: int, torch):
    """Run the fine solver of family member (seed, k) for n_steps coarse steps and
    collect a pair every `every` coarse steps."""
    nf = n_coarse * ratio
    w0, gamma = family_state(seed, k, nf)
    fine_buf = torch.empty((6, nf, nf), dtype=torch.float32, device="cuda")
    a0 = torch.empty((6, n_coarse, n_coarse), dtype=torch.float32, device="cuda")
    with Solver(nx=nf, ny=nf, precision=FP32, gamma=gamma) as fine, \
            Solver(nx=n_coarse, ny=n_coarse, precision=FP32, gamma=gamma) as coarse:
        fine.set_state(w0, None, 0.0)
        fine.set_fixed_dt(dt_c / ratio)
        coarse_steps = 0
        while coarse_steps + 1 <= n_steps:
            fine.get_state_dev(fine_buf)
            block_average(fine_buf, 6, nf, nf, ratio, a0)
            fine.steps(ratio)
            fine.get_state_dev(fine_buf)
            a1 = torch.empty_like(a0)
            block_average(fine_buf, 6, nf, nf, ratio, a1)
            coarse.set_state_dev(a0, None, 0.0)
            coarse.step(dt_c)
            xp = torch.empty_like(a0)
            coarse.get_state_dev(xp)
            pairs.x.append(xp)
            pairs.r.append(a1 - xp)
            pairs.gamma.append(gamma)
            coarse_steps += 1
            skip = min(every - 1, n_steps - coarse_steps)
            if skip > 0:
                fine.steps(ratio * skip)
                coarse_steps += skip
        fine.sync()
    return pairs


def out_scales(pairs: Pairs, torch) -> np.ndarray:
    """Per-field RMS of the residuals (the network predicts residual / scale)."""
    acc = torch.zeros(6, dtype=torch.float64, device="cuda")
    for r in pairs.r:
        acc += (r.double() ** 2).mean(dim=(1, 2))
    rms = torch.sqrt(acc / len(pairs)).cpu().numpy()
    return np.maximum(rms, 1e-30).astype(np.float32)


def train(net: CNN, pairs: Pairs, osc: np.ndarray, dx: float, iters: int, lr: float, torch, seed: int = 0,
          log_every: int = 0):
    """Adam on randomly drawn pairs; lr decays by 10x over the run (cosine)."""
    rng = np.random.default_rng(seed)
    inv = torch.from_numpy(1.0 / osc).cuda().view(6, 1, 1)
    targets = [(r * inv).contiguous() for r in pairs.r]
    losses = []
    for it in range(iters):
        j = int(rng.integers(len(pairs)))
        lr_t = lr * (0.1 + 0.9 * 0.5 * (1 + math.cos(math.pi * it / max(1, iters))))
        want = log_every > 0 and (it % log_every == 0 or it == iters - 1)
        loss = net.train_step(pairs.x[j], targets[j], pairs.gamma[j], dx, dx, lr_t, want_loss=want)
        if want:
            losses.append((it, loss))
    return losses


def residual_gain(net: CNN, pairs: Pairs, osc: np.ndarray, dx: float, torch) -> float:
    """mean |r - out_scale f(x')| / mean |r| over pairs (1 = no gain)."""
    n = pairs.x[0].shape[1]
    pred = torch.empty((n * n, 8), dtype=torch.float32, device="cuda")
    num = den = 0.0
    sc = torch.from_numpy(osc).cuda().view(6, 1, 1)
    for x, r, g in zip(pairs.x, pairs.r, pairs.gamma):
        net.forward(x, g, dx, dx, pred)
        corr = pred[:, :6].t().reshape(6, n, n) * sc
        num += float((r - corr).abs().sum())
        den += float(r.abs().sum())
    return num / den


def run_plain(w0, gamma, n, dt, steps, torch, net=None):
    """Coarse (or plain) run of `steps` fixed steps; with `net`, the correction after
    every step.  Returns the final state (device) and the device time in seconds."""
    out = torch.empty((6, n, n), dtype=torch.float32, device="cuda")
    with Solver(nx=n, ny=n, precision=FP32, gamma=gamma) as s:
        s.set_state(w0, None, 0.0)
        s.set_fixed_dt(dt)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.steps(1)
        if net is not None:
            net.apply(s)
        e0.record(stream)
        if net is None:
            s.steps(steps - 1)
        else:
            for _ in range(steps - 1):
                s.steps(1)
                net.apply(s)
        e1.record(stream)
        e1.synchronize()
        s.sync()
        s.get_state_dev(out)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) * steps / max(1, steps - 1)
    return out, ms * 1e-3


def l1_error(a, b) -> np.ndarray:
    """Relative L1 error per field of a against b (device tensors [6, n, n])."""
    return ((a - b).abs().sum(dim=(1, 2)) / b.abs().sum(dim=(1, 2))).double().cpu().numpy()


def downsample(x, n_to, torch):
    n = x.shape[1]
    r = n // n_to
    if r == 1:
        return x
    out = torch.empty((6, n_to, n_to), dtype=torch.float32, device="cuda")
    block_average(x.contiguous(), 6, n, n, r, out)
    return out


def equal_error_time(curve, err):
    """Log-log interpolation of the plain run time at L1 error `err` on a curve of
    (time, error) points sorted by resolution; None if outside the curve."""
    pts = sorted(curve, key=lambda p: p[0])
    for (t0, e0), (t1, e1) in zip(pts, pts[1:]):
        if (e0 - err) * (e1 - err) <= 0 and e0 != e1:
            a = (math.log(err) - math.log(e0)) / (math.log(e1) - math.log(e0))
            return math.exp(math.log(t0) + a * (math.log(t1) - math.log(t0)))
    return None
