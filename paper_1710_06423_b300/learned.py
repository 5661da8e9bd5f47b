"""Learned coarse-grid correction: data from the fine solver, training, evaluation.

A coarse FP32 run (grid n) takes classical RK4 steps of a fixed size dt_c;
after each step the network of ``sac_cnn_*`` adds its correction
u <- u + out_scale * f(features(u)).  The network is trained on pairs the fine
solver generates: the fine run (grid r*n, step dt_c/r) is block-averaged
(r x r) to the coarse grid at times t_k and t_k + dt_c; the coarse solver
steps the first average once, and the target is the remaining difference to
the second, divided by out_scale.  The plain fine solver is both the source of
the training data and the reference for the error (relative L1 per field against
its block average at the horizon).

Every array operation of the solver and the network runs in the library's CUDA
kernels (solver steps, block averages, network forward/backward/update,
correction); this module sequences the calls and keeps device tensors.  The one
torch arithmetic is the per-step share of an m-step target (a lerp per pair,
training-data preparation only).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs
from .sac import CNN, FP32, SacError, Solver, block_average

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
    """Training pairs on the device: x' (the coarse state after m coarse steps
    from avg(fine(t))) and next, the state the corrected step should reach; the
    network's target (next - x') / out_scale is formed inside the loss kernel.
    With m = 1, next = avg(fine(t + dt_c)).  With m > 1 (substeps), raw =
    avg(fine(t + m dt_c)), and either (share) next = x' + (raw - x') / m, the
    per-step share of the correction the m plain steps missed, for a network
    applied after every step; or (not share) next = raw, the whole missed
    correction, for a network applied after every m-th step (apply_every)."""

    def __init__(self, substeps: int = 1, share: bool = True):
        self.substeps, self.share = substeps, share
        self.apply_every = 1 if share else substeps
        self.x, self.next, self.gamma = [], [], []
        self.raw = []    # avg(fine) at the end of the pair's m steps (= next when m = 1)
        self.meta = []   # (family member, coarse step index of the pair's start)
        self.final = {}  # member -> block-averaged fine state at the horizon (members that reached it)

    def __len__(self):
        return len(self.x)


def _target(pairs: "Pairs", xp, raw, torch):
    """The pair's target: x' + (raw - x') / m (share), else raw."""
    m = pairs.substeps
    return raw if m == 1 or not pairs.share else torch.lerp(xp, raw, 1.0 / m)


def generate_pairs(pairs: Pairs, seed: int, k: int, n_coarse: int, ratio: int, dt_c: float, n_steps: int,
                   every: int, torch, solver_kw=None):
    """Run the fine solver of family member (seed, k) for n_steps coarse steps and
    collect a pair every `every` coarse steps (pairs.substeps coarse steps per
    pair, at most `every`; solver_kw: extra sac_params fields,
    e.g. the diffusion coefficients, used by both grids).  A member that reaches
    the horizon keeps its block-averaged final state in pairs.final[k].  If the
    fine run turns non-finite, the pairs collected before stay and the member
    ends there; returns the number of coarse steps the member completed."""
    kw = dict(solver_kw or {})
    nf = n_coarse * ratio
    m = pairs.substeps
    if not 1 <= m <= every:
        raise ValueError("substeps must be in 1 .. every")
    w0, gamma = family_state(seed, k, nf)
    fine_buf = torch.empty((6, nf, nf), dtype=torch.float32, device="cuda")
    a0 = torch.empty((6, n_coarse, n_coarse), dtype=torch.float32, device="cuda")
    with Solver(nx=nf, ny=nf, precision=FP32, gamma=gamma, **kw) as fine, \
            Solver(nx=n_coarse, ny=n_coarse, precision=FP32, gamma=gamma, **kw) as coarse:
        fine.set_state(w0, None, 0.0)
        fine.set_fixed_dt(dt_c / ratio)
        coarse_steps = 0
        try:
            while coarse_steps + m <= n_steps:
                fine.get_state_dev(fine_buf)
                block_average(fine_buf, 6, nf, nf, ratio, a0)
                fine.steps(ratio * m)
                fine.get_state_dev(fine_buf)
                fine.sync()                      # a non-finite fine state stops here
                a1 = torch.empty_like(a0)
                block_average(fine_buf, 6, nf, nf, ratio, a1)
                coarse.set_state_dev(a0, None, 0.0)
                for _ in range(m):
                    coarse.step(dt_c)
                xp = torch.empty_like(a0)
                coarse.get_state_dev(xp)
                pairs.x.append(xp)
                pairs.next.append(_target(pairs, xp, a1, torch))
                pairs.raw.append(a1)
                pairs.gamma.append(gamma)
                pairs.meta.append((k, coarse_steps))
                coarse_steps += m
                skip = min(every - m, n_steps - coarse_steps)
                if skip > 0:
                    fine.steps(ratio * skip)
                    coarse_steps += skip
            fine.get_state_dev(fine_buf)
            fine.sync()
            final = torch.empty_like(a0)
            block_average(fine_buf, 6, nf, nf, ratio, final)
            pairs.final[k] = final
        except SacError:
            pass
    return coarse_steps


def rollout_pairs(net: CNN, pairs: Pairs, seed: int, members, n_coarse: int, ratio: int, dt_c: float, torch,
                  solver_kw=None) -> Pairs:
    """Pairs on the network's own trajectories (dataset aggregation): for each
    member, the corrected coarse run (the network applied after every step, with
    its current scales and limiter) is started from the block-averaged fine
    initial state (applied every pairs.apply_every steps); at the coarse step of
    each stored pair of that member, its state is stepped pairs.substeps more
    times by the plain coarse solver, and that state is paired with the pair's
    fine target (as Pairs forms it).  The network so also learns to pull
    the states its own rollout reaches back toward the fine solution.  A member
    whose corrected run turns non-finite stops contributing there."""
    kw = dict(solver_kw or {})
    nf = n_coarse * ratio
    m, every = pairs.substeps, pairs.apply_every
    out = Pairs(m, pairs.share)
    for k in members:
        idx = [j for j, (m, _) in enumerate(pairs.meta) if m == k]
        if not idx:
            continue
        at = {pairs.meta[j][1]: j for j in idx}
        w0f, gamma = family_state(seed, k, nf)
        wf = torch.from_numpy(w0f.astype(np.float32)).cuda().contiguous()
        w0c = torch.empty((6, n_coarse, n_coarse), dtype=torch.float32, device="cuda")
        block_average(wf, 6, nf, nf, ratio, w0c)
        del wf
        with Solver(nx=n_coarse, ny=n_coarse, precision=FP32, gamma=gamma, **kw) as roll, \
                Solver(nx=n_coarse, ny=n_coarse, precision=FP32, gamma=gamma, **kw) as one:
            roll.set_state_dev(w0c, None, 0.0)
            roll.set_fixed_dt(dt_c)
            try:
                for step in range(max(at) + 1):
                    if step in at:
                        xr = torch.empty_like(w0c)
                        roll.get_state_dev(xr)
                        one.set_state_dev(xr, None, 0.0)
                        for _ in range(m):
                            one.step(dt_c)
                        one.get_state_dev(xr)
                        j = at[step]
                        out.x.append(xr)
                        out.next.append(_target(pairs, xr, pairs.raw[j], torch))
                        out.raw.append(pairs.raw[j])
                        out.gamma.append(gamma)
                        out.meta.append((k, step))
                    roll.steps(1)
                    if (step + 1) % every == 0:
                        net.apply(roll)
                roll.sync()
            except SacError:
                pass
    return out


def pair_losses(net: CNN, pairs: Pairs, dx: float) -> np.ndarray:
    """The network's loss on each pair (sac_cnn_grads: forward, loss, backward)."""
    out = np.empty(len(pairs))
    for j, (x, nx_, g) in enumerate(zip(pairs.x, pairs.next, pairs.gamma)):
        out[j], _ = net.grads(x, nx_, g, dx, dx)
    return out


def select(pairs: Pairs, keep) -> Pairs:
    out = Pairs(pairs.substeps, pairs.share)
    for j in np.flatnonzero(keep):
        out.x.append(pairs.x[j])
        out.next.append(pairs.next[j])
        out.raw.append(pairs.raw[j])
        out.gamma.append(pairs.gamma[j])
        out.meta.append(pairs.meta[j])
    return out


def merged(a: Pairs, b: Pairs) -> Pairs:
    m = Pairs(a.substeps, a.share)
    for p in (a, b):
        m.x += p.x
        m.next += p.next
        m.raw += p.raw
        m.gamma += p.gamma
        m.meta += p.meta
        m.final.update(p.final)
    return m


def choose_relaxation(net: CNN, finals: dict, osc: np.ndarray, seed: int, members, n_coarse: int, ratio: int,
                      dt_c: float, steps: int, alphas, torch, solver_kw=None, every: int = 1):
    """Relaxation of the applied correction (u <- u + alpha out_scale f, after
    every `every`-th step), chosen on training members: each alpha's corrected
    run of every given member that reached the horizon is compared with that
    member's block-averaged fine state there (finals: member -> that state, as
    Pairs.final holds it; mean relative L1 over the fields); alpha = 0 is the
    plain coarse run.  A run that turns non-finite counts as infinite error.  Leaves the network's
    output scales at alpha_best * osc; returns (alpha_best, {alpha: error})."""
    nf = n_coarse * ratio
    errs = {}
    for alpha in alphas:
        e = []
        for k in members:
            if k not in finals:
                continue
            w0f, gamma = family_state(seed, k, nf)
            wf = _dev(w0f, torch)
            w0c = _host(downsample(wf, n_coarse, torch))
            del wf
            net.set_scales(FEATURE_SCALES, osc * alpha)
            try:
                out, _ = run_plain(w0c, gamma, n_coarse, dt_c, steps, torch, net=net if alpha > 0 else None,
                                   solver_kw=solver_kw, every=every)
                e.append(float(l1_error(out, finals[k]).mean()))
            except SacError:
                e.append(math.inf)
        if e:
            errs[float(alpha)] = float(np.mean(e))
    best = min(errs, key=errs.get) if errs else 0.0
    net.set_scales(FEATURE_SCALES, osc * best)
    return best, errs


def _host(x):
    return x.double().cpu().numpy()


def out_scales(pairs: Pairs, torch, samples: int = 16) -> np.ndarray:
    """Per-field RMS of the residuals next - x' over evenly spaced pairs (host);
    the network predicts residual / scale."""
    idx = np.linspace(0, len(pairs) - 1, min(samples, len(pairs))).astype(int)
    acc = np.zeros(6)
    for j in idx:
        r = _host(pairs.next[j]) - _host(pairs.x[j])
        acc += (r * r).mean(axis=(1, 2))
    return np.maximum(np.sqrt(acc / len(idx)), 1e-30).astype(np.float32)


def train(net: CNN, pairs: Pairs, osc: np.ndarray, dx: float, iters: int, lr: float, torch, seed: int = 0,
          log_every: int = 0, noise: float = 0.0):
    """Adam on randomly drawn pairs; lr decays by 10x over the run (cosine).

    noise > 0: on every other iteration the input x' is perturbed by
    noise * out_scale * U[-1,1) per field (sac_cnn_perturb) while the target state
    stays the fine one, so the network also learns to pull perturbed states back
    (its own errors, in a rollout) toward the fine solution."""
    rng = np.random.default_rng(seed)
    losses = []
    scratch = torch.empty_like(pairs.x[0]) if noise > 0 else None
    amp = (noise * osc).astype(np.float32)
    for it in range(iters):
        j = int(rng.integers(len(pairs)))
        lr_t = lr * (0.1 + 0.9 * 0.5 * (1 + math.cos(math.pi * it / max(1, iters))))
        want = log_every > 0 and (it % log_every == 0 or it == iters - 1)
        x = pairs.x[j]
        if noise > 0 and it % 2 == 1:
            net.perturb(x, scratch, amp, seed * 1000003 + it)
            x = scratch
        loss = net.train_step(x, pairs.next[j], pairs.gamma[j], dx, dx, lr_t, want_loss=want)
        if want:
            losses.append((it, loss))
    return losses


def residual_gain(net: CNN, pairs: Pairs, osc: np.ndarray, dx: float, torch) -> float:
    """mean |r - out_scale f(x')| / mean |r| over pairs, r = next - x' (1 = no gain); host norms."""
    n = pairs.x[0].shape[1]
    pred = torch.empty((n * n, 8), dtype=torch.float32, device="cuda")
    num = den = 0.0
    for x, nx_, g in zip(pairs.x, pairs.next, pairs.gamma):
        net.forward(x, g, dx, dx, pred)
        torch.cuda.synchronize()
        corr = pred.double().cpu().numpy()[:, :6].T.reshape(6, n, n) * osc.astype(np.float64)[:, None, None]
        r = _host(nx_) - _host(x)
        num += float(np.abs(r - corr).sum())
        den += float(np.abs(r).sum())
    return num / den


def run_plain(w0, gamma, n, dt, steps, torch, net=None, solver_kw=None, every: int = 1):
    """Coarse (or plain) run of `steps` fixed steps; with `net`, the correction after
    every `every`-th step.  Returns the final state (device) and the device time in
    seconds (the first `every` steps are untimed; the time is scaled to `steps`)."""
    out = torch.empty((6, n, n), dtype=torch.float32, device="cuda")
    with Solver(nx=n, ny=n, precision=FP32, gamma=gamma, **(solver_kw or {})) as s:
        s.set_state(w0, None, 0.0)
        s.set_fixed_dt(dt)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        first = min(every, steps)
        s.steps(first)
        if net is not None and first == every:
            net.apply(s)
        e0.record(stream)
        if net is None:
            s.steps(steps - first)
        else:
            done = first
            while done < steps:
                k = min(every, steps - done)
                s.steps(k)
                done += k
                if k == every:
                    net.apply(s)
        e1.record(stream)
        e1.synchronize()
        s.sync()
        s.get_state_dev(out)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) * steps / max(1, steps - first)
    return out, ms * 1e-3


def l1_error(a, b) -> np.ndarray:
    """Relative L1 error per field of a against b (device tensors [6, n, n]; host norms)."""
    ah, bh = _host(a), _host(b)
    return np.abs(ah - bh).reshape(6, -1).sum(axis=1) / np.abs(bh).reshape(6, -1).sum(axis=1)


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
