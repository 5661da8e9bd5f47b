"""Gravity about a magnetohydrostatic background (section 2's rho g source):
the CUDA path against the FP64 oracle, the free-fall closed form on the GPU,
and the argument checks."""
import numpy as np
import pytest

from gpu_helpers import TOL_FP32_L1, TOL_FP64, l1rel, maxrel, problem_kwargs

pytestmark = pytest.mark.gpu
G = 2.0


def _case(inputs, nx, ny):
    bg = inputs.stratified_background(nx, ny, g=G, scale_height=0.4, bx=0.3)
    w = np.zeros((6, ny, nx))
    w[0] = inputs.gaussian_blob(nx, ny, amp=0.05, centre=(0.5, 0.45), width=0.12)   # heavy blob
    y = inputs.cell_centres(ny)[:, None] * np.ones((1, nx))
    rho = bg[0] + w[0]
    w[1] = rho * 0.02 * np.sin(2 * np.pi * inputs.cell_centres(nx))[None, :]         # a slow shear flow
    w[3] = 0.5 * w[1] ** 2 / rho + 0.02 * np.exp(-y / 0.4)                          # kinetic + small thermal
    return w, bg


def _kw(nx, ny):
    return problem_kwargs(nx, ny, bc_x=0, bc_y=1, gravity=(0.0, -G))


def _oracle_problem(oracle, kw):
    keys = ("nx", "ny", "x0", "x1", "y0", "y1", "gamma", "courant", "bc_x", "bc_y", "hyperdiffusion", "c2", "c_shk",
            "gravity")
    return oracle.Problem(**{k: kw[k] for k in keys})


@pytest.mark.parametrize("nx,ny,steps", [(40, 56, 6), (70, 33, 4)])
def test_fp64_matches_oracle(oracle_mod, inputs_mod, nx, ny, steps):
    from paper_1710_06423_b300.sac import FP64, Solver
    w, bg = _case(inputs_mod, nx, ny)
    kw = _kw(nx, ny)
    ref, t_ref, n_ref = oracle_mod.run(_oracle_problem(oracle_mod, kw), w, bg=bg, max_steps=steps)
    with Solver(**kw, precision=FP64, has_background=1) as s:
        s.set_state(w, bg, 0.0)
        s.steps(steps)
        got, t = s.get_state()
    assert n_ref == steps and t == pytest.approx(t_ref, rel=0, abs=0)
    assert np.all(maxrel(got, ref) <= TOL_FP64), maxrel(got, ref)


def test_fp32_matches_oracle(oracle_mod, inputs_mod):
    from paper_1710_06423_b300.sac import FP32, Solver
    nx, ny, steps = 96, 80, 40
    w, bg = _case(inputs_mod, nx, ny)
    kw = _kw(nx, ny)
    ref, t_ref, _ = oracle_mod.run(_oracle_problem(oracle_mod, kw), w, bg=bg, max_steps=steps)
    with Solver(**kw, precision=FP32, has_background=1) as s:
        s.set_state(w, bg, 0.0)
        s.steps(steps)
        got, t = s.get_state()
    assert t == pytest.approx(t_ref, rel=1e-6)
    # the velocity fields start near zero: measure m by the L1 norm of the whole momentum
    err = l1rel(got, ref)
    assert err[0] <= TOL_FP32_L1 and err[3] <= TOL_FP32_L1, err
    m_err = np.abs(got[1:3] - ref[1:3]).sum() / np.abs(ref[1:3]).sum()
    assert m_err <= 10 * TOL_FP32_L1, m_err
    # the blob sinks: downward momentum where it started
    assert ref[2][ny * 45 // 100, nx // 2] < 0 and got[2][ny * 45 // 100, nx // 2] < 0


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 2e-6)])
def test_free_fall_on_gpu(precision, tol):
    from paper_1710_06423_b300.sac import Solver
    nx, ny, gam, g = 40, 36, 5 / 3, (0.3, -0.7)
    one = np.ones((ny, nx))
    bg = np.stack([one, one / (gam - 1), 0 * one, 0 * one])
    rt, et0 = 0.5, 0.3
    w = np.stack([rt * one, 0 * one, 0 * one, et0 * one, 0 * one, 0 * one])
    dt, n = 0.01, 5
    with Solver(nx=nx, ny=ny, precision=precision, has_background=1, gravity=g) as s:
        s.set_state(w, bg, 0.0)
        s.set_fixed_dt(dt)
        s.steps(n)
        got, t = s.get_state()
    t = n * dt
    np.testing.assert_allclose(got[1], rt * g[0] * t, rtol=tol)
    np.testing.assert_allclose(got[2], rt * g[1] * t, rtol=tol)
    np.testing.assert_allclose(got[3], et0 + rt * (g[0] ** 2 + g[1] ** 2) * t * t / 2, rtol=tol)
    np.testing.assert_array_equal(got[0], np.float32(rt) if precision else rt)


def test_gravity_argument_checks():
    import torch
    from paper_1710_06423_b300.sac import FP32, Batch, SacError, Solver, step_noalloc
    with pytest.raises(SacError):
        Solver(nx=16, ny=16, precision=FP32, gravity=(0.0, -1.0))          # needs a background
    with pytest.raises(SacError):
        Batch([dict(nx=16, ny=16, has_background=1, gravity=(0.0, -1.0))])
    a = torch.zeros((6, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(SacError):
        step_noalloc(a, torch.empty_like(a), nx=16, ny=16, precision=FP32, gravity=(0.0, -1.0))
