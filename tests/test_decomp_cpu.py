"""The block decomposition (section 3 of the paper: equal blocks, a halo
exchange before every RK stage, the maximum wave speed reduced over all
blocks) on gloo ranks, without a GPU.

Each rank owns one block whose stages are computed by the FP64 oracle
(tests/decomp_oracle_domain.py); the exchange order, the neighbour arithmetic
and the max-reduction are the product's (paper_1710_06423_b300.decomp).  A
stage of a cell reads only cells within 3 of it, so with correct ghosts the
decomposed run equals the single-grid oracle run bit for bit.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, px, py, nx, ny, steps, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from decomp_oracle_domain import OracleDomain
        from paper_1710_06423_b300 import decomp, inputs
        grid = decomp.ProcessGrid(nx, ny, px, py)
        w = inputs.orszag_tang(nx, ny, noise=1e-3, seed=31)
        d = OracleDomain(oracle, grid, rank)
        d.set_state(grid.scatter(w, rank))
        decomp.start_dist(grid, d, rank, dist)
        decomp.step_dist(grid, d, rank, dist, nsteps=steps)
        out.put((rank, d.get_state()[0], d.cx, d.cy))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py,nx,ny", [(2, 1, 20, 14), (1, 2, 17, 22), (2, 2, 19, 16), (4, 1, 26, 9)],
                         ids=["2x1", "1x2", "2x2", "4x1"])
def test_decomposed_oracle_run_equals_single_grid(oracle_mod, inputs_mod, px, py, nx, ny):
    import torch.multiprocessing as mp
    from paper_1710_06423_b300 import decomp
    steps = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29400 + (os.getpid() * 7 + px * 10 + py) % 1000
    world = px * py
    procs = [ctx.Process(target=_worker, args=(r, world, port, px, py, nx, ny, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    grid = decomp.ProcessGrid(nx, ny, px, py)
    got = grid.gather({r: w for r, w, _, _ in res})
    w0 = inputs_mod.orszag_tang(nx, ny, noise=1e-3, seed=31)
    ref, _, n = oracle_mod.run(oracle_mod.Problem(nx=nx, ny=ny), w0, max_steps=steps)
    assert n == steps
    assert np.array_equal(got, ref), np.abs(got - ref).max()
    # every rank holds the global signal speeds of the final state
    cx, cy = oracle_mod.cmax(oracle_mod.Problem(nx=nx, ny=ny), ref)
    assert all(r[2] == cx and r[3] == cy for r in res)


def test_process_grid_neighbours_and_split():
    from paper_1710_06423_b300 import decomp
    g = decomp.ProcessGrid(30, 9, 3, 2)
    # inner block boundaries on multiples of the 4-cell sweep segment
    assert g.xs == [(0, 8), (8, 12), (20, 10)] and g.ys == [(0, 4), (4, 5)]
    assert g.neighbor(0, decomp.LEFT) == 2 and g.neighbor(2, decomp.RIGHT) == 0
    assert g.neighbor(1, decomp.BOTTOM) == 4 and g.neighbor(4, decomp.TOP) == 1
    assert g.phases() == [(decomp.LEFT, decomp.RIGHT), (decomp.BOTTOM, decomp.TOP)]
    w = np.arange(6 * 9 * 30, dtype=float).reshape(6, 9, 30)
    assert np.array_equal(g.gather({r: g.scatter(w, r) for r in range(6)}), w)
    for n, parts in ((97, 2), (130, 3), (26, 4), (1000, 7)):
        sp = decomp.split(n, parts)
        assert sum(c for _, c in sp) == n and all(s0 % 4 == 0 for s0, _ in sp)
    with pytest.raises(ValueError):
        decomp.ProcessGrid(6, 8, 2, 1)          # a block of 2 cells cannot feed a 3-cell halo
    with pytest.raises(ValueError):
        g.local_bc(1, 0)                        # a split direction must be periodic
