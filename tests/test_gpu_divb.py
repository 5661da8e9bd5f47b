"""The device div B diagnostic (sac_divb) against the oracle's discrete div B
of the same stored state: max |div B|, mean |div B| and the count of cells
whose stencil exists, for both precisions, periodic and non-periodic sides,
with and without a background, before and after steps.  With hyper-diffusion
off the central differences commute, so the divergence the device reports
stays where it started.  The 3D form's sums and div B (sac3_sums, sac3_divb)
are checked the same way against sums of the stored state and the oracle's
3D div B."""
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


# ---- the 3D form: sac3_sums and sac3_divb against the oracle ----------------------

def _ot3_noisy(inputs, nx, ny, nz, seed):
    w = inputs.ot_3d(nx, ny, nz, compress=0.3)
    rng = np.random.default_rng(seed)
    w[5:8] += 1e-3 * rng.standard_normal((3, nz, ny, nx))
    return w


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,ny,nz", [(40, 24, 20), (33, 17, 9)])
def test_3d_sums_and_divb_match_oracle(oracle_mod, inputs_mod, precision, nx, ny, nz):
    from paper_1710_06423_b300.sac import FP32, FP64, Solver3
    prec = FP64 if precision == "fp64" else FP32
    w = _ot3_noisy(inputs_mod, nx, ny, nz, seed=nx + nz)
    box = dict(x1=1.0, y1=0.8, z1=1.3)
    pr = oracle_mod.Problem3(nx=nx, ny=ny, nz=nz, **box)
    with Solver3(nx=nx, ny=ny, nz=nz, precision=prec, **box) as s:
        s.set_state(w, 0.0)
        for _ in range(2):
            got, _ = s.get_state()
            sums = s.sums()
            want = got.reshape(8, -1).sum(axis=1)
            scale = np.abs(got).reshape(8, -1).sum(axis=1)
            assert np.all(np.abs(sums - want) <= 1e-12 * scale), (sums, want)
            div = np.abs(oracle_mod.div_b3(pr, got))
            mx, mean = s.divb()
            assert mx == pytest.approx(div.max(), rel=TOL_DIVB, abs=0)
            assert mean == pytest.approx(div.mean(), rel=TOL_DIVB, abs=0)
            assert s.divb() == (mx, mean)
            s.steps(2)


def test_3d_divb_carried_without_hyperdiffusion(inputs_mod):
    from paper_1710_06423_b300.sac import FP64, Solver3
    n = 24
    w = _ot3_noisy(inputs_mod, n, n, n, seed=3)
    with Solver3(nx=n, ny=n, nz=n, precision=FP64, hyperdiffusion=0) as s:
        s.set_state(w, 0.0)
        m0, a0 = s.divb()
        s.steps(10)
        m1, a1 = s.divb()
    assert m0 > 0.05
    assert m1 == pytest.approx(m0, rel=1e-10) and a1 == pytest.approx(a0, rel=1e-10)


def test_3d_diagnostics_need_a_state():
    from paper_1710_06423_b300.sac import FP32, SAC_ERR_STATE, SacError, Solver3
    with Solver3(nx=8, ny=8, nz=8, precision=FP32) as s:
        for call in (s.sums, s.divb):
            with pytest.raises(SacError) as err:
                call()
            assert err.value.code == SAC_ERR_STATE


def test_divb_keeps_a_nan(inputs_mod):
    """A NaN in B shows in both outputs (a plain fmax would drop it from the maximum)."""
    import math
    from paper_1710_06423_b300.sac import FP32, FP64, Solver, Solver3
    n = 40
    w = _noisy_ot(inputs_mod, n, n, seed=1)
    w[4, 17, 23] = np.nan
    for prec in (FP64, FP32):
        with Solver(**problem_kwargs(n, n), precision=prec) as s:
            s.set_state(w, None, 0.0)
            mx, mean, _ = s.divb()
        assert math.isnan(mx) and math.isnan(mean)
    w3 = _ot3_noisy(inputs_mod, 16, 16, 16, seed=2)
    w3[7, 3, 4, 5] = np.nan
    with Solver3(nx=16, ny=16, nz=16, precision=FP32) as s3:
        s3.set_state(w3, 0.0)
        mx, mean = s3.divb()
    assert math.isnan(mx) and math.isnan(mean)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_3d_sums_conserved_on_the_periodic_box(inputs_mod, precision, tol):
    """Flux-form differences on a periodic box conserve every field's sum: the
    device sums after several steps equal the starting sums (to rounding)."""
    from paper_1710_06423_b300.sac import FP32, FP64, Solver3
    prec = FP64 if precision == "fp64" else FP32
    n = 20
    w = _ot3_noisy(inputs_mod, n, n, n, seed=6)
    with Solver3(nx=n, ny=n, nz=n, precision=prec) as s:
        s.set_state(w, 0.0)
        s0 = s.sums()
        scale = np.abs(s.get_state()[0]).reshape(8, -1).sum(axis=1)
        s.steps(6)
        s1 = s.sums()
    assert np.all(np.abs(s1 - s0) <= tol * scale), (s1 - s0) / scale
