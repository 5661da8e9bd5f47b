"""Batched runs (many independent grids, one launch per RK stage) against
single-run contexts and the oracle."""
import numpy as np
import pytest

from gpu_helpers import TOL_FP32_L1, l1rel, oracle_problem, problem_kwargs

pytestmark = pytest.mark.gpu
FP32 = 1


def _family_run(inputs, n, k, seed=2024):
    b0, gamma, phases = inputs.ot_family_params(seed, k)
    w = inputs.orszag_tang(n, b0=b0, gamma=gamma, phases=phases)
    return dict(nx=n, ny=n, gamma=gamma), w


def _single(kw, w, steps):
    from paper_1710_06423_b300.sac import Solver
    with Solver(**kw, precision=FP32) as s:
        s.set_state(w, None, 0.0)
        s.steps(steps)
        return s.get_state()


SIZES = [70, 33, 96, 40, 64]


@pytest.fixture(scope="module")
def small_batch(inputs_mod):
    runs, states = [], []
    for k, n in enumerate(SIZES):
        kw, w = _family_run(inputs_mod, n, k)
        runs.append(kw)
        states.append(w)
    return runs, states


@pytest.mark.parametrize("config", [(1, 2, 0), (1, 1, 2), (0, 2, 1), (2, 2, 1), (2, 1, 2)])
def test_batch_equals_single_runs_bitwise(small_batch, config):
    from paper_1710_06423_b300.sac import Batch
    runs, states = small_batch
    steps = 7
    with Batch(runs) as b:
        b.set_config(*config)
        for i, w in enumerate(states):
            b.set_state(i, w, None, 0.0)
        b.steps(steps)
        b.sync()
        got = [b.get_state(i) for i in range(len(runs))]
    for i, (kw, w) in enumerate(zip(runs, states)):
        ref, tr = _single(kw, w, steps)
        assert got[i][1] == tr
        assert np.array_equal(got[i][0], ref), i


@pytest.mark.parametrize("config", [(2, 2, 0), (2, 2, 2), (1, 2, 2)])
def test_many_tiles_per_cta_equal_single_runs_bitwise(inputs_mod, config):
    """More tiles than resident CTAs, so each persistent CTA walks several tiles
    across run boundaries (arguments reused within a run, reloaded on a change,
    one signal-speed fold per run change in stage 4)."""
    from paper_1710_06423_b300.sac import Batch
    sizes = [1000, 33, 130, 512, 70, 260]
    runs, states = [], []
    for k, n in enumerate(sizes):
        kw, w = _family_run(inputs_mod, n, k, seed=77)
        runs.append(kw)
        states.append(w)
    steps = 3
    with Batch(runs) as b:
        b.set_config(*config)
        for i, w in enumerate(states):
            b.set_state(i, w, None, 0.0)
        b.steps(steps)
        b.sync()
        got = [b.get_state(i) for i in range(len(runs))]
    for i, (kw, w) in enumerate(zip(runs, states)):
        ref, tr = _single(kw, w, steps)
        assert got[i][1] == tr, i
        assert np.array_equal(got[i][0], ref), i


def test_bad_config_rejected(small_batch):
    from paper_1710_06423_b300.sac import SAC_ERR_ARG, Batch, SacError
    runs, _ = small_batch
    with Batch(runs) as b:
        for cfg in ((3, 2, 0), (-1, 2, 0), (1, 3, 0), (1, 2, 3)):
            with pytest.raises(SacError) as err:
                b.set_config(*cfg)
            assert err.value.code == SAC_ERR_ARG


def test_batch_runs_keep_their_own_step(small_batch):
    """Each run takes its own CFL step: times differ across runs of different gamma / B0."""
    from paper_1710_06423_b300.sac import Batch
    runs, states = small_batch
    with Batch(runs) as b:
        for i, w in enumerate(states):
            b.set_state(i, w, None, 0.0)
        b.steps(3)
        times = [b.time(i) for i in range(len(runs))]
    assert all(n == 3 for _, n in times)
    assert len({t for t, _ in times}) > 1


def test_batch_matches_oracle(oracle_mod, small_batch):
    from paper_1710_06423_b300.sac import Batch
    runs, states = small_batch
    steps = 5
    with Batch(runs) as b:
        for i, w in enumerate(states):
            b.set_state(i, w, None, 0.0)
        b.steps(steps)
        got = [b.get_state(i)[0] for i in range(len(runs))]
    for i in (0, 1, 3):
        kw = problem_kwargs(runs[i]["nx"], runs[i]["ny"], gamma=runs[i]["gamma"])
        ref, _, _ = oracle_mod.run(oracle_problem(oracle_mod, kw), states[i], max_steps=steps)
        assert np.all(l1rel(got[i], ref) <= TOL_FP32_L1), (i, l1rel(got[i], ref))


def test_tuner_keeps_states(small_batch):
    """The autotuner advances trial steps and then restores every run exactly."""
    from paper_1710_06423_b300.sac import Batch
    runs, states = small_batch
    with Batch(runs) as b:
        for i, w in enumerate(states):
            b.set_state(i, w, None, 0.0)
        b.steps(2)
        before = [b.get_state(i) for i in range(len(runs))]
        cfg, ms = b.tune(trials=2)
        after = [b.get_state(i) for i in range(len(runs))]
        b.steps(3)
        cont = [b.get_state(i)[0] for i in range(len(runs))]
    assert ms > 0 and cfg[0] in (0, 1, 2) and cfg[1] in (1, 2) and cfg[2] in (0, 1, 2)
    for x, y in zip(before, after):
        assert np.array_equal(x[0], y[0]) and x[1] == y[1]
    for i, (kw, w) in enumerate(zip(runs, states)):
        ref, _ = _single(kw, w, 5)
        assert np.array_equal(cont[i], ref), i


def test_family_batch_shape(inputs_mod):
    """The 64-run family workload: seeded sizes from {256, 512, 1000, 2044}; a few steps of the
    whole batch, with two runs compared bitwise against single-run contexts."""
    from paper_1710_06423_b300.sac import Batch
    sizes = inputs_mod.batch_sizes(2024, 64)
    assert set(sizes) <= {256, 512, 1000, 2044} and len(set(sizes)) >= 3
    runs, states = [], []
    for k, n in enumerate(sizes):
        kw, w = _family_run(inputs_mod, n, k)
        runs.append(kw)
        states.append(w)
    with Batch(runs) as b:
        for i, w in enumerate(states):
            b.set_state(i, w, None, 0.0)
        b.tune(trials=1)
        b.steps(4)
        b.sync()
        picks = [sizes.index(256), sizes.index(512)]
        got = {i: b.get_state(i) for i in picks}
    for i in picks:
        ref, tr = _single(runs[i], states[i], 4)
        assert np.array_equal(got[i][0], ref) and got[i][1] == tr


@pytest.mark.parametrize("config", [(1, 2, 1), (2, 2, 0), (0, 2, 2)])
def test_batch_with_background_and_open_sides_equals_single_runs(config):
    """Runs with a static background and fixed/outflow/periodic sides (the
    background instantiation of the batch kernel and the non-periodic ghost
    frames): bit for bit the same as single-run contexts."""
    from gpu_helpers import smooth_background
    from paper_1710_06423_b300.sac import Batch, Solver
    import paper_1710_06423_b300.inputs as inputs
    cases = [(70, 45, 0, 2), (96, 64, 2, 1), (33, 90, 1, 0), (128, 40, 2, 2)]
    runs, states = [], []
    for k, (nx, ny, bx, by) in enumerate(cases):
        bg = smooth_background(ny, nx, seed=k + 1)
        w = inputs.orszag_tang(nx, ny, noise=1e-3, seed=k)
        w[0] += 0.3 - bg[0]
        w[3] += 0.5 - bg[1]
        w[4] -= bg[2]
        w[5] -= bg[3]
        runs.append(dict(nx=nx, ny=ny, bc_x=bx, bc_y=by, has_background=1))
        states.append((w, bg))
    steps = 4
    with Batch(runs) as b:
        b.set_config(*config)
        for i, (w, bg) in enumerate(states):
            b.set_state(i, w, bg, 0.0)
        b.steps(steps)
        b.sync()
        got = [b.get_state(i) for i in range(len(runs))]
    for i, (kw, (w, bg)) in enumerate(zip(runs, states)):
        with Solver(**kw, precision=FP32) as s:
            s.set_state(w, bg, 0.0)
            s.steps(steps)
            ref, t = s.get_state()
        assert got[i][1] == t, i
        assert np.array_equal(got[i][0], ref), i


@pytest.mark.parametrize("config", [(1, 2, 2), (2, 2, 1), (0, 2, 0)])
def test_batch_with_one_row_and_tiny_runs_equals_single_runs(config):
    """Degenerate grids in one batch: the Brio-Wu tube (800 x 1, fixed sides,
    gamma 2), a 5 x 3 periodic grid, a 1 x 40 column and a multi-tile run."""
    from paper_1710_06423_b300.sac import Batch, Solver
    import paper_1710_06423_b300.inputs as inputs
    runs = [dict(nx=800, ny=1, gamma=2.0, bc_x=1, bc_y=1),
            dict(nx=5, ny=3),
            dict(nx=1, ny=40, bc_y=2),
            dict(nx=100, ny=70)]
    states = [inputs.brio_wu(800, 1, gamma=2.0),
              inputs.orszag_tang(5, 3, noise=1e-3, seed=3),
              inputs.orszag_tang(1, 40, noise=1e-3, seed=4),
              inputs.orszag_tang(100, 70, noise=1e-3, seed=5)]
    steps = 5
    with Batch(runs) as b:
        b.set_config(*config)
        for i, w in enumerate(states):
            b.set_state(i, w, None, 0.0)
        b.steps(steps)
        b.sync()
        got = [b.get_state(i) for i in range(len(runs))]
    for i, (kw, w) in enumerate(zip(runs, states)):
        with Solver(**kw, precision=FP32) as s:
            s.set_state(w, None, 0.0)
            s.steps(steps)
            ref, t = s.get_state()
        assert got[i][1] == t, i
        assert np.array_equal(got[i][0], ref), i
