"""Pins of the oracle's gravity source terms (no GPU).

Section 2 adds rho g to the momentum equation and its work to the energy
equation; with the background read as magnetohydrostatic (its own weight
balanced), the perturbation sources are rt g and m.g.  The pins:

* free fall: a uniform perturbation density rt on a uniform background, at
  rest, accelerates as a whole.  Fluxes stay uniform and hyper-diffusion
  vanishes, so m = rt g t and et = et0 + rt |g|^2 t^2 / 2 exactly (classical RK4
  integrates these polynomials in t without error).  A source written with the
  total density, a wrong sign, a missing energy term or the kinetic energy
  taken from the wrong density each break it;
* a balanced stratified background with a zero perturbation stays exactly
  zero under gravity (the background's weight is not counted twice).
"""
import numpy as np
import pytest

BC_P, BC_F, BC_O = 0, 1, 2


@pytest.mark.parametrize("g", [(0.0, -0.7), (0.3, -0.7), (-0.45, 0.2)])
def test_free_fall_closed_form(oracle_mod, g):
    o = oracle_mod
    nx, ny, gam = 12, 10, 5 / 3
    pr = o.Problem(nx=nx, ny=ny, gamma=gam, gravity=g, hyperdiffusion=1)
    one = np.ones((ny, nx))
    bg = np.stack([1.0 * one, (1.0 / (gam - 1)) * one, 0.0 * one, 0.0 * one])   # rho_b, e_b, B_b
    rt, et0 = 0.5, 0.3
    w = np.stack([rt * one, 0 * one, 0 * one, et0 * one, 0 * one, 0 * one])
    dt, n = 0.01, 5
    out, t, steps = o.run(pr, w, bg=bg, max_steps=n, fixed_dt=dt)
    assert steps == n
    t = n * dt
    np.testing.assert_array_equal(out[0], w[0])                       # density untouched
    np.testing.assert_allclose(out[1], rt * g[0] * t, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(out[2], rt * g[1] * t, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(out[3], et0 + rt * (g[0] ** 2 + g[1] ** 2) * t * t / 2, rtol=1e-13)
    np.testing.assert_array_equal(out[4:], 0.0)


def test_balanced_stratified_background_stays_at_rest(oracle_mod, inputs_mod):
    o = oracle_mod
    nx, ny = 16, 24
    g = 2.0
    pr = o.Problem(nx=nx, ny=ny, gravity=(0.0, -g), bc_x=BC_P, bc_y=BC_F, hyperdiffusion=1)
    bg = inputs_mod.stratified_background(nx, ny, g=g, scale_height=0.4, bx=0.3, gamma=pr.gamma)
    w = np.zeros((6, ny, nx))
    out, t, steps = o.run(pr, w, bg=bg, max_steps=4, fixed_dt=1e-3)
    assert steps == 4
    np.testing.assert_array_equal(out, 0.0)
    # the same background with a heavy blob: the blob's own momentum turns downward
    w[0] = inputs_mod.gaussian_blob(nx, ny, amp=0.05, centre=(0.5, 0.5), width=0.1)
    k = o.rhs(pr, w, bg=bg, cmax=o.cmax(pr, w, bg))
    c = (ny // 2, nx // 2)
    assert k[2][c] < 0.0 and k[2][c] == pytest.approx(w[0][c] * -g, rel=1e-12)
