"""Stream binding: a context runs on the CUDA stream it was created with
(captured graphs are replayed there).  The same run gives the same bits on
torch's current stream, on a side stream and on the legacy default stream,
and two contexts stepped in turn on two side streams (their work enqueued
back to back, then synchronised) each give their own serial result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(kw, w, steps, stream):
    from paper_1710_06423_b300.sac import FP32, Solver
    with Solver(**kw, precision=FP32, stream=stream) as s:
        s.set_state(w, None, 0.0)
        s.steps(steps)
        return s.get_state()


def test_same_bits_on_every_stream(inputs_mod):
    import torch
    kw = dict(nx=130, ny=70)
    w = inputs_mod.orszag_tang(130, 70, noise=1e-3, seed=21)
    ref, t = _run(kw, w, 12, "current")
    side = torch.cuda.Stream()
    for stream in (side, None):
        got, t2 = _run(kw, w, 12, stream)
        assert t2 == t and np.array_equal(got, ref)


def test_two_contexts_interleaved_on_two_streams(inputs_mod):
    import torch
    from paper_1710_06423_b300.sac import FP32, Solver
    kws = [dict(nx=200, ny=96), dict(nx=96, ny=150, bc_x=2)]
    ws = [inputs_mod.orszag_tang(200, 96, noise=1e-3, seed=1), inputs_mod.orszag_tang(96, 150, noise=1e-3, seed=2)]
    want = [_run(kw, w, 10, "current") for kw, w in zip(kws, ws)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    solvers = [Solver(**kw, precision=FP32, stream=st) for kw, st in zip(kws, streams)]
    try:
        for s, w in zip(solvers, ws):
            s.set_state(w, None, 0.0)
        for _ in range(5):                      # enqueue both runs' steps in turn
            for s in solvers:
                s.steps(2)
        for s in solvers:
            s.sync()
        for s, (ref, t) in zip(solvers, want):
            got, t2 = s.get_state()
            assert t2 == t and np.array_equal(got, ref)
    finally:
        for s in solvers:
            s.close()
