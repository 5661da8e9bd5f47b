"""Tile shapes of the FP32 stage kernel and their autotuner.

Every shape (32 x 32, 64 x 16, 32 x 16 cells), with the ghost frame written by
a separate kernel or by the stage kernel itself, must give bit for bit the
results of the default 32 x 32 tiles: a cell's arithmetic is the same whatever
tile it falls in, and the ghost cells receive the same copies, so only the work
distribution changes.  Checked on ragged grids
(several tiles plus partial ones in both directions), with every boundary
kind, with a background, in single runs and in batches; one non-default shape
is also compared with the oracle directly.  The tuner must restore the state
it advanced, keep the fastest shape and hand it to later contexts of the same
configuration.
"""
import numpy as np
import pytest

from gpu_helpers import TOL_FP32_L1, l1rel, oracle_problem, problem_kwargs, smooth_background

pytestmark = pytest.mark.gpu
FP32 = 1
SHAPES = (0, 1, 2)   # SAC_TILE_32x32, SAC_TILE_64x16, SAC_TILE_32x16
CONFIGS = SHAPES + (3, 4, 5)   # the same shapes with the in-kernel ghost frame

CASES = [
    # nx, ny, kwargs, background
    (70, 45, {}, False),
    (130, 37, {"bc_x": 2, "bc_y": 1}, False),
    (97, 66, {"bc_y": 2}, True),
    (33, 1, {}, False),
    (1, 40, {"bc_y": 2}, False),
    (200, 150, {"hyperdiffusion": 0}, False),
    # for the in-kernel ghost frame (grids narrower than the 3-cell frame are
    # the 33 x 1 and 1 x 40 cases): a fixed side beside a periodic one, last
    # tiles narrower than the frame, outflow on both sides
    (66, 70, {"bc_x": 1}, False),
    (65, 34, {}, False),
    (35, 19, {"bc_x": 2, "bc_y": 2}, False),
]


def _state(inputs, nx, ny, has_bg):
    w = inputs.orszag_tang(nx, ny, noise=1e-3, seed=13)
    bg = None
    if has_bg:
        bg = smooth_background(ny, nx)
        w = w.copy()
        w[0] -= bg[0] - 0.3
        w[3] -= bg[1] - 0.5
        w[4] -= bg[2]
        w[5] -= bg[3]
    return w, bg


def _run(kw, w, bg, tile, steps):
    from paper_1710_06423_b300.sac import Solver
    with Solver(**kw, precision=FP32, has_background=int(bg is not None)) as s:
        s.set_tile(tile)
        assert s.tile() == tile
        s.set_state(w, bg, 0.0)
        s.steps(steps)
        return s.get_state()


@pytest.mark.parametrize("nx,ny,kw,has_bg", CASES, ids=[f"{c[0]}x{c[1]}" for c in CASES])
def test_every_tile_shape_equals_the_default_bitwise(inputs_mod, nx, ny, kw, has_bg):
    kw = problem_kwargs(nx, ny, **kw)
    w, bg = _state(inputs_mod, nx, ny, has_bg)
    ref, t_ref = _run(kw, w, bg, 0, 6)
    for tile in CONFIGS[1:]:
        got, t = _run(kw, w, bg, tile, 6)
        assert t == t_ref
        assert np.array_equal(got, ref), (tile, np.abs(got - ref).max())


def test_non_default_tile_against_the_oracle(oracle_mod, inputs_mod):
    kw = problem_kwargs(150, 90)
    w, _ = _state(inputs_mod, 150, 90, False)
    ref, t_ref, _ = oracle_mod.run(oracle_problem(oracle_mod, kw), w, max_steps=10)
    for tile in (1, 2, 4):
        got, t = _run(kw, w, None, tile, 10)
        assert abs(t - t_ref) <= 1e-6 * t_ref
        assert np.all(l1rel(got, ref) <= TOL_FP32_L1), (tile, l1rel(got, ref))


def test_tuner_restores_the_state_and_keeps_the_fastest_shape(inputs_mod):
    from paper_1710_06423_b300.sac import Solver
    n = 300
    kw = problem_kwargs(n, n)
    w, _ = _state(inputs_mod, n, n, False)
    with Solver(**kw, precision=FP32) as s:
        s.set_state(w, None, 0.0)
        s.steps(2)
        before, t0 = s.get_state()
        tile, ms = s.tune(trials=2)
        after, t1 = s.get_state()
        assert tile in CONFIGS and ms > 0 and s.tile() == tile
        assert t1 == t0 and s.time() == (t0, 2)
        assert np.array_equal(after, before)
        s.steps(3)
        got, _ = s.get_state()
    ref, _ = _run(kw, w, None, 0, 5)
    assert np.array_equal(got, ref)
    # a later context of the same configuration starts with the tuned shape
    with Solver(**kw, precision=FP32) as s2:
        assert s2.tile() == tile


def test_tile_api_rejects_bad_shapes_and_fp64(inputs_mod):
    from paper_1710_06423_b300.sac import FP64, SacError, Solver
    with Solver(nx=16, ny=16, precision=FP32) as s:
        for bad in (-1, 6):
            with pytest.raises(SacError):
                s.set_tile(bad)
    with Solver(nx=16, ny=16, precision=FP64) as s:
        with pytest.raises(SacError):
            s.set_tile(1)


@pytest.mark.parametrize("tile", [1, 2])
@pytest.mark.parametrize("config", [(1, 2, 1), (2, 2, 2), (0, 2, 0), (1, 1, 0)])
def test_batch_tile_shapes_equal_single_runs_bitwise(inputs_mod, tile, config):
    from paper_1710_06423_b300.sac import Batch, Solver
    sizes = [1000, 33, 130, 257, 70]
    runs, states = [], []
    for k, n in enumerate(sizes):
        b0, gamma, phases = inputs_mod.ot_family_params(55, k)
        runs.append(dict(nx=n, ny=n, gamma=gamma))
        states.append(inputs_mod.orszag_tang(n, b0=b0, gamma=gamma, phases=phases))
    steps = 3
    with Batch(runs) as b:
        b.set_config(*config)
        b.set_tile(tile)
        assert b.config() == (*config, tile)
        for i, w in enumerate(states):
            b.set_state(i, w, None, 0.0)
        b.steps(steps)
        b.sync()
        got = [b.get_state(i) for i in range(len(runs))]
    for i, (kw, w) in enumerate(zip(runs, states)):
        with Solver(**kw, precision=FP32) as s:
            s.set_state(w, None, 0.0)
            s.steps(steps)
            ref, tr = s.get_state()
        assert got[i][1] == tr, i
        assert np.array_equal(got[i][0], ref), (i, sizes[i])


def test_batch_tuner_reports_a_tile_shape(inputs_mod):
    from paper_1710_06423_b300.sac import Batch
    sizes = [256, 512, 256]
    runs, states = [], []
    for k, n in enumerate(sizes):
        b0, gamma, phases = inputs_mod.ot_family_params(56, k)
        runs.append(dict(nx=n, ny=n, gamma=gamma))
        states.append(inputs_mod.orszag_tang(n, b0=b0, gamma=gamma, phases=phases))
    with Batch(runs) as b:
        for i, w in enumerate(states):
            b.set_state(i, w, None, 0.0)
        before = [b.get_state(i) for i in range(len(runs))]
        cfg, ms = b.tune(trials=1)
        full = b.config()
        assert full[:3] == cfg and full[3] in SHAPES and ms > 0
        for i in range(len(runs)):
            g, t = b.get_state(i)
            assert t == before[i][1] and np.array_equal(g, before[i][0])
