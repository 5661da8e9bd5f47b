"""The allocation-free step (sac_step_noalloc) against the allocating one.

Some callers cannot allocate device memory (for example a plug-in whose host
application owns all device memory through its own allocator, or a real-time
loop where an allocation's device synchronisation and unbounded latency are not
allowed); for them the library keeps the working memory of one FP32 RK4 step in
a fixed array compiled into it.  This test calls that entry point through the C ABI twice in a row,
each time on the previous output, and checks it against the context-based path
(sac_set_state_dev + sac_step + sac_get_state_dev) on the same states.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import TOL_FP32_L1, l1rel

pytestmark = pytest.mark.gpu


def test_noalloc_step_matches_context_step_twice(inputs_mod):
    import torch
    from paper_1710_06423_b300 import sac
    nx, ny = 200, 150
    w0 = inputs_mod.orszag_tang(nx, ny, noise=1e-3, seed=9)
    dev = torch.from_numpy(w0.astype(np.float32)).cuda().contiguous()
    # reference: the context path, two CFL steps
    refs, dts = [], []
    with sac.Solver(nx=nx, ny=ny, precision=sac.FP32) as s:
        s.set_state_dev(dev, None, 0.0)
        for _ in range(2):
            dts.append(s.step(0.0))
            r = torch.empty_like(dev)
            s.get_state_dev(r)
            torch.cuda.synchronize()
            refs.append(r.double().cpu().numpy())
    # the allocation-free path, two calls in a row
    a = dev.clone()
    b = torch.empty_like(dev)
    dt1 = sac.step_noalloc(a, b, 0.0, nx=nx, ny=ny)
    dt2 = sac.step_noalloc(b, a, 0.0, nx=nx, ny=ny)
    torch.cuda.synchronize()
    got = [b.double().cpu().numpy(), a.double().cpu().numpy()]
    assert (dt1, dt2) == tuple(dts)
    for g, r in zip(got, refs):
        assert np.all(l1rel(g, r) <= TOL_FP32_L1), l1rel(g, r)
        assert np.array_equal(g, r)          # same kernels, same arithmetic


@pytest.mark.parametrize("case", ["brio_wu_fixed", "outflow", "in_place"])
def test_noalloc_edge_cases_equal_context_step(inputs_mod, case):
    """The 1D Brio-Wu tube with fixed sides (held ghosts taken from the input
    state, as sac_set_state takes them), an outflow grid, and an in-place call
    (w_out == w_in): bit for bit the context path's step."""
    import torch
    from paper_1710_06423_b300 import sac
    if case == "brio_wu_fixed":
        kw = dict(nx=800, ny=1, gamma=2.0, bc_x=1, bc_y=1)
        w0 = inputs_mod.brio_wu(800, 1, gamma=2.0)
    else:
        kw = dict(nx=37, ny=29, bc_x=2, bc_y=2) if case == "outflow" else dict(nx=64, ny=48)
        w0 = inputs_mod.orszag_tang(kw["nx"], kw["ny"], noise=1e-3, seed=2)
    dev = torch.from_numpy(w0.astype(np.float32)).cuda().contiguous()
    with sac.Solver(**kw, precision=sac.FP32) as s:
        s.set_state_dev(dev, None, 0.0)
        dt_ref = s.step(0.0)
        ref = torch.empty_like(dev)
        s.get_state_dev(ref)
    a = dev.clone()
    b = a if case == "in_place" else torch.empty_like(dev)
    dt = sac.step_noalloc(a, b, 0.0, **kw)
    torch.cuda.synchronize()
    assert dt == dt_ref
    assert torch.equal(b, ref)


def test_noalloc_fixed_step_equals_context_step(inputs_mod):
    """A given step size (dt > 0) goes through the step-begin override instead
    of the CFL step: two such calls in a row equal Solver.step(dt) bit for bit."""
    import torch
    from paper_1710_06423_b300 import sac
    nx, ny = 96, 80
    w0 = inputs_mod.orszag_tang(nx, ny, noise=1e-3, seed=4)
    dev = torch.from_numpy(w0.astype(np.float32)).cuda().contiguous()
    dt = 1.25e-3
    refs = []
    with sac.Solver(nx=nx, ny=ny, precision=sac.FP32) as s:
        s.set_state_dev(dev, None, 0.0)
        for _ in range(2):
            assert s.step(dt) == dt
            r = torch.empty_like(dev)
            s.get_state_dev(r)
            refs.append(r.clone())
    a, b = dev.clone(), torch.empty_like(dev)
    assert sac.step_noalloc(a, b, dt, nx=nx, ny=ny) == dt
    assert sac.step_noalloc(b, a, dt, nx=nx, ny=ny) == dt
    torch.cuda.synchronize()
    assert torch.equal(b, refs[0]) and torch.equal(a, refs[1])


def test_noalloc_rejects_grids_beyond_its_memory():
    import torch
    from paper_1710_06423_b300 import sac
    w = torch.zeros((6, 300, 300), dtype=torch.float32, device="cuda")
    with pytest.raises(sac.SacError) as ei:
        sac.step_noalloc(w, w, 0.0, nx=300, ny=300)
    assert ei.value.code == sac.SAC_ERR_TOO_LARGE
