"""Pins of the 3D oracle (no GPU).

* A z-uniform state with m_z = B_z = 0 evolves exactly as the 2D oracle does
  (each z term of the 3D sums is an exact zero added last): bitwise, over
  several CFL steps, with the z extent chosen so that dz/cmax_z is not the
  smallest step.
* The same with x and z exchanged: an x-uniform state in the (y, z) plane
  reproduces the 2D run with (x, y) -> (y, z) (checks the z operator itself).
* Fourth-order convergence of an oblique linear sound wave.
* Periodic sums of all eight fields are conserved.
"""
import math

import numpy as np
import pytest


def _to3d_z(w2, nz):
    """2D state (6, ny, nx) -> z-uniform 3D state (8, nz, ny, nx) with m_z = B_z = 0."""
    r, mx, my, e, bx, by = w2
    z = np.zeros_like(r)
    f = [r, mx, my, z, e, bx, by, z]
    return np.ascontiguousarray(np.stack([np.broadcast_to(a, (nz,) + a.shape) for a in f]))


def test_z_uniform_equals_2d(oracle_mod, inputs_mod):
    o = oracle_mod
    nx, ny, nz = 20, 16, 3
    w2 = inputs_mod.orszag_tang(nx, ny, noise=1e-3, seed=7)
    pr2 = o.Problem(nx=nx, ny=ny, c2=(0.02, 0.1, 0.1, 0.02, 0.02, 0.02))
    pr3 = o.Problem3(nx=nx, ny=ny, nz=nz, z1=100.0)
    ref, t2, _ = o.run(pr2, w2, max_steps=4)
    got, t3, _ = o.run3(pr3, _to3d_z(w2, nz), max_steps=4)
    assert t3 == t2
    for kz in range(nz):
        np.testing.assert_array_equal(got[[0, 1, 2, 4, 5, 6], kz], ref)
    np.testing.assert_array_equal(got[3], 0.0)
    np.testing.assert_array_equal(got[7], 0.0)


def test_x_uniform_equals_2d_in_yz(oracle_mod, inputs_mod):
    o = oracle_mod
    ny, nz, nx = 16, 20, 3
    w2 = inputs_mod.orszag_tang(ny, nz, noise=1e-3, seed=9)    # 2D (x, y) -> 3D (y, z)
    r, m1, m2, e, b1, b2 = w2
    z = np.zeros_like(r)
    f = [r, z, m1, m2, e, z, b1, b2]
    w3 = np.ascontiguousarray(np.stack([np.broadcast_to(a[:, :, None], (nz, ny, nx)) for a in f]))
    pr2 = o.Problem(nx=ny, ny=nz, c2=(0.02, 0.1, 0.1, 0.02, 0.02, 0.02))
    pr3 = o.Problem3(nx=nx, ny=ny, nz=nz, x1=100.0)
    ref, t2, _ = o.run(pr2, w2, max_steps=3)
    got, t3, _ = o.run3(pr3, w3, max_steps=3)
    assert t3 == t2
    for kx in range(nx):
        np.testing.assert_array_equal(got[[0, 2, 3, 4, 6, 7], :, :, kx], ref)


def test_oblique_sound_wave_fourth_order(oracle_mod):
    """rho = 1 + a sin(2 pi (x + y + z)), small amplitude: error against the exact
    travelling wave after a fixed time falls by ~2^4 per refinement."""
    o = oracle_mod
    amp, gam, T = 1e-10, 5 / 3, 0.05
    errs = []
    for n in (8, 16):
        c = (np.arange(n) + 0.5) / n
        X, Y, Z = np.meshgrid(c, c, c, indexing="xy")
        X, Y, Z = np.transpose(X, (2, 0, 1)), np.transpose(Y, (2, 0, 1)), np.transpose(Z, (2, 0, 1))
        ph = 2 * math.pi * (X + Y + Z)
        cs = 1.0                                  # p0 = 1/gamma, rho0 = 1
        kdir = np.array([1, 1, 1]) / math.sqrt(3)
        w = np.zeros((8, n, n, n))
        s = np.sin(ph)
        w[0] = 1 + amp * s
        for q in range(3):
            w[1 + q] = amp * s * cs * kdir[q]
        w[4] = (1 / gam + gam * (1 / gam) * amp * s) / (gam - 1)
        pr = o.Problem3(nx=n, ny=n, nz=n, hyperdiffusion=0)
        steps = 8 * n
        out, t, _ = o.run3(pr, w, max_steps=steps, fixed_dt=T / steps)
        exact = 1 + amp * np.sin(ph - 2 * math.pi * math.sqrt(3) * cs * T)
        errs.append(np.abs(out[0] - exact).max() / amp)
    assert errs[0] / errs[1] > 12, errs


def test_periodic_sums_conserved(oracle_mod):
    o = oracle_mod
    n = 10
    rng = np.random.default_rng(3)
    w = np.zeros((8, n, n, n))
    w[0] = 1 + 0.1 * rng.random((n, n, n))
    w[1:4] = 0.05 * rng.standard_normal((3, n, n, n))
    w[5:8] = 0.1 * rng.standard_normal((3, n, n, n))
    w[4] = 2.0 + 0.5 * (w[5:8] ** 2).sum(axis=0)
    pr = o.Problem3(nx=n, ny=n, nz=n)
    out, _, _ = o.run3(pr, w, max_steps=3)
    s0, s1 = w.reshape(8, -1).sum(axis=1), out.reshape(8, -1).sum(axis=1)
    np.testing.assert_allclose(s1, s0, rtol=0, atol=1e-12 * np.abs(w).reshape(8, -1).sum(axis=1).max())


def test_one_step_depends_only_on_cells_within_12(oracle_mod, inputs_mod):
    """One RK4 step reads 3 cells per stage in every direction, so the step on a
    periodically-wrapped window with a 12-cell margin equals the full-grid step
    inside the margin (the basis of the full-size window parity test)."""
    o = oracle_mod
    n, size, margin = 48, 8, 12
    m = size + 2 * margin
    w = inputs_mod.ot_3d(n, n, n, compress=0.4)
    pr = o.Problem3(nx=n, ny=n, nz=n)
    cm = o.cmax3(pr, w)
    dt = o.cfl_dt3(pr, *cm)
    full = o.rk4_step3(pr, w, dt, cm)
    ref_run, _, _ = o.run3(pr, w, max_steps=1)
    np.testing.assert_array_equal(full, ref_run)
    for k0, j0, i0 in [(0, 0, 0), (40, 3, 45), (20, 30, 10)]:
        idx = [np.arange(q - margin, q + size + margin) % n for q in (k0, j0, i0)]
        win = np.ascontiguousarray(w[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]])
        # the window's grid spacing is exactly 1/n (m/n and (m/n)/m are exact here)
        prw = o.Problem3(nx=m, ny=m, nz=m, x1=m / n, y1=m / n, z1=m / n)
        got = o.rk4_step3(prw, win, dt, cm)[:, margin:-margin, margin:-margin, margin:-margin]
        inner = [np.arange(q, q + size) % n for q in (k0, j0, i0)]
        exp = full[:, inner[0]][:, :, inner[1]][:, :, :, inner[2]]
        np.testing.assert_array_equal(got, exp)
