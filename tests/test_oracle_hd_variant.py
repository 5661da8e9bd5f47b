"""Pins of the single-face hyper-diffusion variant (no maximum over three faces;
stencil radius 2) against closed forms (no GPU).

With R_f = |d3_f| / |d1_f| on the face itself the face flux is
nu_f d1_f = c2 dx cmax sign(d1_f) |d3_f| (c_shk = 0):
* a cubic a + b i^3 has d3 = 6b on every face and d1_f > 0, so the flux is
  constant and the diffusion term vanishes (the three-face form does not);
* a quartic b i^4 has d3_f = 12 b (2f + 1), d1_f > 0 for f >= 0, so the
  diffusion term is the constant 24 c2 cmax b / dx.
"""
import numpy as np

BC_O = 2


def _uniform(nx):
    from paper_1710_06423_b300.inputs import conserved
    o = np.ones((1, nx))
    return conserved(o, 0 * o, 0 * o, o, 0 * o, 0 * o, 5 / 3)


def test_cubic_gives_zero(oracle_mod):
    o = oracle_mod
    nx, b, c2, cm = 30, 2.0 ** -13, 0.07, 1.7
    i = np.arange(nx, dtype=float)
    w = _uniform(nx)
    w[0, 0] = 1.0 + b * i ** 3
    single = o.Problem(nx=nx, ny=1, bc_x=BC_O, c2=(c2, 0, 0, 0, 0, 0), c_shk=0.0, hd_single_face=1)
    triple = o.Problem(nx=nx, ny=1, bc_x=BC_O, c2=(c2, 0, 0, 0, 0, 0), c_shk=0.0, hd_single_face=0)
    k1 = o.rhs(single, w, cmax=(cm, 0.0))[0, 0, 4:nx - 4]
    k3 = o.rhs(triple, w, cmax=(cm, 0.0))[0, 0, 4:nx - 4]
    scale = c2 * cm * 6 * b / single.dx
    assert np.all(np.abs(k1) <= 1e-12 * scale)
    assert np.all(np.abs(k3) > 1e-3 * scale)          # the three-face form does diffuse


def test_quartic_closed_form(oracle_mod):
    o = oracle_mod
    nx, b, c2, cm = 30, 2.0 ** -20, 0.05, 1.3
    i = np.arange(nx, dtype=float)
    w = _uniform(nx)
    w[0, 0] = 1.0 + b * i ** 4
    pr = o.Problem(nx=nx, ny=1, bc_x=BC_O, c2=(c2, 0, 0, 0, 0, 0), c_shk=0.0, hd_single_face=1)
    k = o.rhs(pr, w, cmax=(cm, 0.0))[0, 0, 4:nx - 4]
    np.testing.assert_allclose(k, 24 * c2 * cm * b / pr.dx, rtol=1e-10)


def test_single_face_conserves_periodic_sums(oracle_mod, inputs_mod):
    o = oracle_mod
    n = 24
    pr = o.Problem(nx=n, ny=n, hd_single_face=1)
    w = inputs_mod.orszag_tang(n)
    out, t, steps = o.run(pr, w, max_steps=3)
    s0 = w.reshape(6, -1).sum(axis=1)
    s1 = out.reshape(6, -1).sum(axis=1)
    np.testing.assert_allclose(s1, s0, rtol=0, atol=1e-12 * np.abs(w).reshape(6, -1).sum(axis=1).max())
