"""The block decomposition on the GPU: px x py blocks of one grid, each an
ordinary context stepped stage by stage (sac_stage) with its 3-cell halo strips
moved between blocks (sac_halo_pack / sac_halo_unpack) before every stage and
the signal-speed keys reduced with a maximum after every step.  The blocks run
in one process on one GPU (host-ordered stages; no kernel waits on another), so
this exercises the library's half of a multi-GPU run: with correct ghosts, the
same cell size and the global signal speeds the decomposed run equals the
single-grid run bit for bit, in FP32 and FP64.
"""
import numpy as np
import pytest

from gpu_helpers import problem_kwargs

pytestmark = pytest.mark.gpu
FP64, FP32 = 0, 1


@pytest.mark.parametrize("precision", [FP32, FP64], ids=["fp32", "fp64"])
@pytest.mark.parametrize("px,py,nx,ny,kw", [
    (2, 1, 70, 45, {}),
    (1, 2, 70, 45, {}),
    (2, 2, 97, 66, {}),
    (3, 2, 130, 37, {}),
    (2, 1, 64, 33, {"bc_y": 2}),          # split in x, outflow in y
    (1, 3, 41, 90, {"bc_x": 1}),          # split in y, fixed in x
], ids=["2x1", "1x2", "2x2", "3x2", "2x1_outflow_y", "1x3_fixed_x"])
def test_decomposed_run_equals_single_grid_bitwise(inputs_mod, precision, px, py, nx, ny, kw):
    from paper_1710_06423_b300 import decomp
    from paper_1710_06423_b300.sac import Solver
    steps = 5
    params = problem_kwargs(nx, ny, **kw)
    w0 = inputs_mod.orszag_tang(nx, ny, noise=1e-3, seed=17)
    with Solver(**params, precision=precision) as s:
        s.set_state(w0, None, 0.0)
        s.steps(steps)
        ref, t_ref = s.get_state()
        cref = s.cmax()
    grid = decomp.ProcessGrid(nx, ny, px, py)
    bparams = {k: v for k, v in params.items() if k not in ("nx", "ny")}
    doms = {r: decomp.CudaDomain(grid, r, precision=precision, **bparams) for r in range(grid.size)}
    try:
        for r, d in doms.items():
            d.set_state(grid.scatter(w0, r))
        decomp.start_local(grid, doms)
        decomp.step_local(grid, doms, steps)
        parts, times = {}, set()
        for r, d in doms.items():
            w, t = d.get_state()
            parts[r] = w
            times.add(t)
            assert d.solver.cmax() == cref
        got = grid.gather(parts)
    finally:
        for d in doms.values():
            d.close()
    assert times == {t_ref}
    assert np.array_equal(got, ref), np.abs(got - ref).max()


def test_stage_order_and_halo_arguments_are_checked(inputs_mod):
    import torch
    from paper_1710_06423_b300.sac import FP32 as P32, SacError, Solver
    with Solver(nx=16, ny=16, precision=P32, bc_x=1) as s:
        s.set_state(inputs_mod.orszag_tang(16, 16), None, 0.0)
        with pytest.raises(SacError):
            s.stage(2)                       # stages come in order
        s.stage(1)
        with pytest.raises(SacError):
            s.step(0.0)                      # a half-done step blocks the other stepping calls
        for k in (2, 3, 4):
            s.stage(k)
        assert s.halo_size(0) == 6 * 3 * 22 and s.halo_size(3) == 6 * 22 * 3
        with pytest.raises(SacError):
            s.halo_size(4)
        s.step(0.0)
    with Solver(nx=2, ny=16, precision=P32) as s:
        with pytest.raises(SacError):
            s.halo_size(0)                   # fewer than 3 cells across the strip
