"""Pins of the oracle's discrete div B (section 2's fourth-order central
difference applied to the total field B = B_b + B~).

* closed form: on a periodic grid the five-point difference of sin(a x) is
  a cos(a x) times the scheme's modified-wavenumber factor
  (8 sin(a h) - sin(2 a h)) / (6 a h), and likewise for cos(b y);
* polynomial exactness: the difference is exact for polynomials of degree
  four or less, so on outflow sides the counted cells give the analytic
  divergence to rounding;
* mask: a non-periodic side leaves out the two cells next to it, a periodic
  side none, a direction of one cell none;
* split invariance: moving part of B into the background changes nothing;
* a field built from a discrete vector potential with the same difference
  (Bx = D_y A, By = -D_x A) has zero divergence, which fails if the x and y
  derivatives were swapped or a component taken from the wrong field.

The 3D form's div B (Dx Bx + Dy By + Dz Bz on a periodic box) is pinned the
same way: the closed form with a different wavenumber per axis, a z-uniform
field equal to the 2D divergence in every plane, and zero for the discrete
curl of a vector potential (fails for exchanged components).
"""
import numpy as np
import pytest


def _zero_state(n_x, n_y):
    return np.zeros((6, n_y, n_x))


def test_divb_closed_form_sines(oracle_mod):
    o = oracle_mod
    nx, ny = 40, 24
    pr = o.Problem(nx=nx, ny=ny, x0=0.0, x1=2.0, y0=-1.0, y1=0.5)
    x = pr.x0 + (np.arange(nx) + 0.5) * pr.dx
    y = pr.y0 + (np.arange(ny) + 0.5) * pr.dy
    a = 2 * np.pi * 3 / (pr.x1 - pr.x0)
    b = 2 * np.pi * 2 / (pr.y1 - pr.y0)
    w = _zero_state(nx, ny)
    w[4] = 0.7 * np.sin(a * x)[None, :]
    w[5] = 1.3 * np.cos(b * y)[:, None]
    div, mask = o.div_b(pr, w)
    assert mask.all()

    def factor(k, h):
        return (8 * np.sin(k * h) - np.sin(2 * k * h)) / (6 * k * h)

    want = (0.7 * a * factor(a, pr.dx) * np.cos(a * x)[None, :]
            - 1.3 * b * factor(b, pr.dy) * np.sin(b * y)[:, None])
    np.testing.assert_allclose(div, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_divb_exact_for_quartics_on_outflow_sides(oracle_mod):
    o = oracle_mod
    nx, ny = 17, 13
    pr = o.Problem(nx=nx, ny=ny, x0=-0.5, x1=1.2, y0=0.0, y1=0.9, bc_x=o.BC_OUTFLOW, bc_y=o.BC_FIXED)
    x = pr.x0 + (np.arange(nx) + 0.5) * pr.dx
    y = pr.y0 + (np.arange(ny) + 0.5) * pr.dy
    w = _zero_state(nx, ny)
    w[4] = (x ** 4 - x ** 3 + 0.5 * x)[None, :] * np.ones((ny, 1))
    w[5] = (y ** 2 - 3 * y ** 4)[:, None] * np.ones((1, nx))
    div, mask = o.div_b(pr, w)
    want = (4 * x ** 3 - 3 * x ** 2 + 0.5)[None, :] + (2 * y - 12 * y ** 3)[:, None]
    assert mask.sum() == (nx - 4) * (ny - 4)
    assert not mask[:, :2].any() and not mask[:, -2:].any() and not mask[:2].any() and not mask[-2:].any()
    np.testing.assert_allclose(div[mask], want[mask], rtol=0, atol=1e-11)
    assert np.all(div[~mask] == 0.0)


def test_divb_mask_rules(oracle_mod):
    o = oracle_mod
    w = np.random.default_rng(1).standard_normal((6, 9, 11))
    _, m = o.div_b(o.Problem(nx=11, ny=9), w)
    assert m.all()
    _, m = o.div_b(o.Problem(nx=11, ny=9, bc_x=o.BC_OUTFLOW), w)
    assert m.sum() == 7 * 9 and m[:, 2:9].all()
    _, m = o.div_b(o.Problem(nx=11, ny=9, bc_y=o.BC_FIXED), w)
    assert m.sum() == 11 * 5 and m[2:7].all()
    # one row: the y term is absent and no row is left out
    w1 = np.random.default_rng(2).standard_normal((6, 1, 20))
    pr1 = o.Problem(nx=20, ny=1, bc_x=o.BC_OUTFLOW, bc_y=o.BC_OUTFLOW)
    d1, m1 = o.div_b(pr1, w1)
    assert m1.sum() == 16
    bx = w1[4, 0]
    i = 7
    want = (bx[i - 2] - 8 * bx[i - 1] + 8 * bx[i + 1] - bx[i + 2]) / (12 * pr1.dx)
    assert d1[0, i] == pytest.approx(want, rel=1e-14)


def test_divb_split_invariance(oracle_mod):
    o = oracle_mod
    rng = np.random.default_rng(3)
    nx, ny = 20, 16
    pr = o.Problem(nx=nx, ny=ny, bc_y=o.BC_OUTFLOW)
    w = rng.standard_normal((6, ny, nx))
    bg = np.zeros((4, ny, nx))
    bg[0] = 1.0
    bg[2] = rng.standard_normal((ny, nx))
    bg[3] = rng.standard_normal((ny, nx))
    d_split, m_split = o.div_b(pr, w, bg)
    w_tot = w.copy()
    w_tot[4] += bg[2]
    w_tot[5] += bg[3]
    d_tot, m_tot = o.div_b(pr, w_tot)
    assert np.array_equal(m_split, m_tot)
    np.testing.assert_allclose(d_split, d_tot, rtol=0, atol=1e-12 * np.abs(d_tot).max())
    # a non-zero background divergence is seen
    d_pert, _ = o.div_b(pr, w)
    assert np.abs(d_split - d_pert).max() > 1.0


def test_divb_zero_for_discrete_vector_potential(oracle_mod):
    o = oracle_mod
    nx, ny = 24, 20
    pr = o.Problem(nx=nx, ny=ny, x1=3.0, y1=2.0)
    A = np.random.default_rng(4).standard_normal((ny, nx))

    def five_point(f, axis, h):
        return ((np.roll(f, 2, axis) - np.roll(f, -2, axis)) + 8 * (np.roll(f, -1, axis) - np.roll(f, 1, axis))) / (12 * h)

    w = _zero_state(nx, ny)
    w[4] = five_point(A, 0, pr.dy)      # Bx = dA/dy
    w[5] = -five_point(A, 1, pr.dx)     # By = -dA/dx
    div, _ = o.div_b(pr, w)
    scale = np.abs(w[4]).max() / pr.dx
    assert np.abs(div).max() < 1e-12 * scale
    # the same field with the components exchanged is far from solenoidal
    w2 = w.copy()
    w2[4], w2[5] = w[5].copy(), w[4].copy()
    div2, _ = o.div_b(pr, w2)
    assert np.abs(div2).max() > 1e-2 * scale


# ---- the 3D form: div B = Dx Bx + Dy By + Dz Bz on a periodic box ----------------

def test_divb3_closed_form_sines(oracle_mod):
    o = oracle_mod
    nx, ny, nz = 20, 12, 16
    pr = o.Problem3(nx=nx, ny=ny, nz=nz, x1=2.0, y0=-1.0, y1=0.5, z1=0.8)
    h = ((pr.x1 - pr.x0) / nx, (pr.y1 - pr.y0) / ny, (pr.z1 - pr.z0) / nz)
    x = pr.x0 + (np.arange(nx) + 0.5) * h[0]
    y = pr.y0 + (np.arange(ny) + 0.5) * h[1]
    z = pr.z0 + (np.arange(nz) + 0.5) * h[2]
    a = 2 * np.pi * 3 / (pr.x1 - pr.x0)
    b = 2 * np.pi * 2 / (pr.y1 - pr.y0)
    c = 2 * np.pi * 1 / (pr.z1 - pr.z0)
    w = np.zeros((8, nz, ny, nx))
    w[5] = 0.7 * np.sin(a * x)[None, None, :]
    w[6] = 1.3 * np.cos(b * y)[None, :, None]
    w[7] = -0.4 * np.sin(c * z + 0.3)[:, None, None]

    def factor(k, hh):
        return (8 * np.sin(k * hh) - np.sin(2 * k * hh)) / (6 * k * hh)

    want = (0.7 * a * factor(a, h[0]) * np.cos(a * x)[None, None, :]
            - 1.3 * b * factor(b, h[1]) * np.sin(b * y)[None, :, None]
            - 0.4 * c * factor(c, h[2]) * np.cos(c * z + 0.3)[:, None, None])
    div = o.div_b3(pr, w)
    np.testing.assert_allclose(div, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_divb3_z_uniform_equals_2d(oracle_mod):
    o = oracle_mod
    nx, ny, nz = 14, 10, 6
    rng = np.random.default_rng(8)
    b2 = rng.standard_normal((2, ny, nx))
    w3 = np.zeros((8, nz, ny, nx))
    w3[5] = b2[0][None]
    w3[6] = b2[1][None]
    w3[7] = 0.37                       # a uniform B_z has no z derivative
    w2 = np.zeros((6, ny, nx))
    w2[4], w2[5] = b2
    d3 = o.div_b3(o.Problem3(nx=nx, ny=ny, nz=nz, x1=1.5, y1=0.7), w3)
    d2, m2 = o.div_b(o.Problem(nx=nx, ny=ny, x1=1.5, y1=0.7), w2)
    assert m2.all()
    for k in range(nz):
        np.testing.assert_allclose(d3[k], d2, rtol=0, atol=1e-13 * np.abs(d2).max())


def test_divb3_zero_for_discrete_curl(oracle_mod):
    o = oracle_mod
    nx, ny, nz = 12, 10, 8
    pr = o.Problem3(nx=nx, ny=ny, nz=nz, x1=1.2, y1=0.9, z1=2.0)
    h = (pr.x1 / nx, pr.y1 / ny, pr.z1 / nz)
    A = np.random.default_rng(9).standard_normal((3, nz, ny, nx))

    def D(f, axis):   # axis 2: x, 1: y, 0: z of a [nz][ny][nx] array
        hh = h[2 - axis]
        return ((np.roll(f, 2, axis) - np.roll(f, -2, axis)) + 8 * (np.roll(f, -1, axis) - np.roll(f, 1, axis))) / (12 * hh)

    w = np.zeros((8, nz, ny, nx))
    w[5] = D(A[2], 1) - D(A[1], 0)     # Bx = dAz/dy - dAy/dz
    w[6] = D(A[0], 0) - D(A[2], 2)     # By = dAx/dz - dAz/dx
    w[7] = D(A[1], 2) - D(A[0], 1)     # Bz = dAy/dx - dAx/dy
    scale = np.abs(w[5:]).max() / min(h)
    assert np.abs(o.div_b3(pr, w)).max() < 1e-12 * scale
    w2 = w.copy()
    w2[5], w2[7] = w[7].copy(), w[5].copy()
    assert np.abs(o.div_b3(pr, w2)).max() > 1e-2 * scale
