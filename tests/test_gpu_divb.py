"""The device div B diagnostic (sac_divb) against the oracle's discrete div B
of the same stored state: max |div B|, mean |div B| and the count of cells
whose stencil exists, for both precisions, periodic and non-periodic sides,
with and without a background, before and after steps.  With hyper-diffusion
off the central differences commute, so the divergence the device reports
stays where it started."""
import numpy as np
import pytest

from gpu_helpers import oracle_problem, problem_kwargs, smooth_background

pytestmark = pytest.mark.gpu

TOL_DIVB = 1e-12   # FP64 on both sides; only the rounding of 1/(12h) and the summation order differ


def _noisy_ot(inputs, nx, ny, seed):
    w = inputs.orszag_tang(nx, ny, noise=1e-3, seed=seed)
    rng = np.random.default_rng(seed + 100)
    w[4] += 1e-3 * rng.standard_normal((ny, nx))     # a non-zero discrete div B
    w[5] += 1e-3 * rng.standard_normal((ny, nx))
    return w


def _check(oracle, kw, s, bg):
    got, _ = s.get_state()
    div, mask = oracle.div_b(oracle_problem(oracle, kw), got, bg)
    want_max = np.abs(div[mask]).max()
    want_mean = np.abs(div[mask]).mean()
    mx, mean, n = s.divb()
    assert n == int(mask.sum())
    assert mx == pytest.approx(want_max, rel=TOL_DIVB, abs=0)
    assert mean == pytest.approx(want_mean, rel=TOL_DIVB, abs=0)
    return mx, mean


CASES = [
    # nx, ny, bc_x, bc_y, background
    (150, 90, 0, 0, False),
    (97, 131, 2, 1, True),
    (64, 48, 0, 2, True),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,ny,bcx,bcy,has_bg", CASES)
def test_divb_matches_oracle(oracle_mod, inputs_mod, precision, nx, ny, bcx, bcy, has_bg):
    from paper_1710_06423_b300.sac import FP32, FP64, Solver
    prec = FP64 if precision == "fp64" else FP32
    w = _noisy_ot(inputs_mod, nx, ny, seed=nx)
    bg = smooth_background(ny, nx, seed=ny) if has_bg else None
    if bg is not None:
        w[0] += 0.3            # keep total density and pressure comfortably positive
        w[3] += 0.5
        if prec == FP32:
            bg = bg.astype(np.float32).astype(np.float64)   # the FP32 context stores the background in FP32
    kw = problem_kwargs(nx, ny, bc_x=bcx, bc_y=bcy)
    with Solver(**kw, precision=prec, has_background=int(has_bg)) as s:
        s.set_state(w, bg, 0.0)
        m0, _ = _check(oracle_mod, kw, s, bg)
        assert m0 > 0.05
        s.steps(3)
        _check(oracle_mod, kw, s, bg)
        a, b = s.divb(), s.divb()
        assert a == b                                  # fixed reduction order


def test_divb_one_row(oracle_mod, inputs_mod):
    from paper_1710_06423_b300.sac import FP64, Solver
    n = 300
    w = inputs_mod.brio_wu(n, 1, gamma=2.0)
    w[4] += 1e-3 * np.random.default_rng(7).standard_normal((1, n))
    kw = problem_kwargs(n, 1, gamma=2.0, bc_x=2, bc_y=2)
    with Solver(**kw, precision=FP64) as s:
        s.set_state(w, None, 0.0)
        _, _ = _check(oracle_mod, kw, s, None)
        assert s.divb()[2] == n - 4


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 2e-3)])
def test_divb_carried_without_hyperdiffusion(inputs_mod, precision, tol):
    from paper_1710_06423_b300.sac import FP32, FP64, Solver
    prec = FP64 if precision == "fp64" else FP32
    n = 128
    w = _noisy_ot(inputs_mod, n, n, seed=11)
    kw = problem_kwargs(n, n, hyperdiffusion=0)
    with Solver(**kw, precision=prec) as s:
        s.set_state(w, None, 0.0)
        m0, a0, _ = s.divb()
        s.steps(20)
        m1, a1, _ = s.divb()
    assert m1 == pytest.approx(m0, rel=tol) and a1 == pytest.approx(a0, rel=tol)


def test_divb_needs_a_state():
    from paper_1710_06423_b300.sac import FP32, SAC_ERR_STATE, SacError, Solver
    with Solver(nx=16, ny=16, precision=FP32) as s:
        with pytest.raises(SacError) as err:
            s.divb()
        assert err.value.code == SAC_ERR_STATE
