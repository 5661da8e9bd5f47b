"""The 3D form on the GPU against the FP64 3D oracle (and, for z-uniform
states, against the 2D solver)."""
import numpy as np
import pytest

from gpu_helpers import TOL_FP32_L1, TOL_FP64, l1rel, maxrel

pytestmark = pytest.mark.gpu


def _rel(a, b):
    n = a.shape[0]
    return maxrel(a.reshape(n, -1), b.reshape(n, -1))


@pytest.mark.parametrize("nx,ny,nz,steps", [(12, 10, 8, 3), (16, 16, 16, 2)])
def test_fp64_matches_oracle(oracle_mod, inputs_mod, nx, ny, nz, steps):
    from paper_1710_06423_b300.sac import FP64, Solver3
    w = inputs_mod.ot_3d(nx, ny, nz)
    pr = oracle_mod.Problem3(nx=nx, ny=ny, nz=nz)
    ref, t_ref, _ = oracle_mod.run3(pr, w, max_steps=steps)
    with Solver3(nx=nx, ny=ny, nz=nz, precision=FP64) as s:
        s.set_state(w, 0.0)
        s.steps(steps)
        got, t = s.get_state()
    assert t == t_ref
    assert np.all(_rel(got, ref) <= TOL_FP64), _rel(got, ref)


# FP32 cases span several 32 x 4 column tiles and 32-plane z chunks of the fused
# kernel with ragged tails, an anisotropic box, hyper-diffusion off, and a
# compressive flow that switches the shock viscosity on.
FP32_CASES = [
    dict(n=(24, 24, 24), steps=10, kw={}, compress=0.0),
    dict(n=(37, 11, 70), steps=4, kw=dict(x1=1.5, z1=2.0), compress=0.3),
    dict(n=(33, 9, 40), steps=4, kw=dict(hyperdiffusion=0), compress=0.3),
    dict(n=(64, 8, 33), steps=3, kw=dict(y1=0.5), compress=0.5),
    dict(n=(45, 13, 37), steps=5, kw=dict(z1=1.3), compress=0.4),
    dict(n=(12, 12, 12), steps=6, kw={}, compress=0.3),
]


@pytest.mark.parametrize("case", FP32_CASES, ids=lambda c: "x".join(map(str, c["n"])) + str(c["kw"]))
def test_fp32_matches_oracle(oracle_mod, inputs_mod, case):
    from paper_1710_06423_b300.sac import FP32, Solver3
    nx, ny, nz = case["n"]
    steps = case["steps"]
    w = inputs_mod.ot_3d(nx, ny, nz, compress=case["compress"])
    pr = oracle_mod.Problem3(nx=nx, ny=ny, nz=nz, **case["kw"])
    ref, t_ref, _ = oracle_mod.run3(pr, w, max_steps=steps)
    with Solver3(nx=nx, ny=ny, nz=nz, precision=FP32, **case["kw"]) as s:
        s.set_state(w, 0.0)
        s.steps(steps)
        got, t = s.get_state()
    assert t == pytest.approx(t_ref, rel=1e-5)
    err = l1rel(got.reshape(8, -1), ref.reshape(8, -1))
    assert np.all(err <= TOL_FP32_L1), err


def test_fp64_compressive_matches_oracle(oracle_mod, inputs_mod):
    from paper_1710_06423_b300.sac import FP64, Solver3
    nx, ny, nz = 20, 9, 14
    w = inputs_mod.ot_3d(nx, ny, nz, compress=0.5)
    pr = oracle_mod.Problem3(nx=nx, ny=ny, nz=nz, y1=0.7)
    ref, t_ref, _ = oracle_mod.run3(pr, w, max_steps=3)
    with Solver3(nx=nx, ny=ny, nz=nz, y1=0.7, precision=FP64) as s:
        s.set_state(w, 0.0)
        s.steps(3)
        got, t = s.get_state()
    assert t == t_ref
    assert np.all(_rel(got, ref) <= TOL_FP64), _rel(got, ref)


def test_z_uniform_matches_2d_solver(inputs_mod):
    from paper_1710_06423_b300.sac import FP64, Solver, Solver3
    nx, ny, nz = 40, 24, 2
    w2 = inputs_mod.orszag_tang(nx, ny, noise=1e-3, seed=11)
    r, mx, my, e, bx, by = w2
    z = np.zeros_like(r)
    w3 = np.ascontiguousarray(np.stack([np.broadcast_to(a, (nz, ny, nx)) for a in (r, mx, my, z, e, bx, by, z)]))
    with Solver(nx=nx, ny=ny, precision=FP64, c2=(0.02, 0.1, 0.1, 0.02, 0.02, 0.02)) as s2:
        s2.set_state(w2, None, 0.0)
        s2.steps(3)
        ref, t2 = s2.get_state()
    with Solver3(nx=nx, ny=ny, nz=nz, z1=100.0, precision=FP64) as s3:
        s3.set_state(w3, 0.0)
        s3.steps(3)
        got, t3 = s3.get_state()
    assert t3 == t2
    for kz in range(nz):
        assert np.all(maxrel(got[[0, 1, 2, 4, 5, 6], kz], ref) <= TOL_FP64)


def test_nonfinite_state_is_reported():
    from paper_1710_06423_b300.sac import FP32, SacError, Solver3
    n = 8
    w = np.zeros((8, n, n, n))
    w[0] = -1.0                                   # negative density: no real signal speed
    w[4] = 1.0
    with Solver3(nx=n, ny=n, nz=n, precision=FP32) as s:
        s.set_state(w, 0.0)
        with pytest.raises(SacError):
            s.step()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,ny,nz", [(40, 24, 1), (1, 30, 20), (17, 1, 9)])
def test_one_cell_thick_boxes_match_oracle(oracle_mod, inputs_mod, precision, nx, ny, nz):
    """Degenerate boxes (one cell along z, x or y): the periodic wrap of a
    single plane, row or column, against the 3D oracle."""
    from paper_1710_06423_b300.sac import FP32, FP64, Solver3
    prec = FP64 if precision == "fp64" else FP32
    steps = 3
    w = inputs_mod.ot_3d(nx, ny, nz, compress=0.3)
    pr = oracle_mod.Problem3(nx=nx, ny=ny, nz=nz)
    ref, t_ref, _ = oracle_mod.run3(pr, w, max_steps=steps)
    with Solver3(nx=nx, ny=ny, nz=nz, precision=prec) as s:
        s.set_state(w, 0.0)
        s.steps(steps)
        got, t = s.get_state()
    live = [f for f in range(8) if np.abs(ref[f]).sum() > 0]
    for f in range(8):
        if f not in live:
            assert np.abs(got[f]).max() <= (0.0 if prec == FP64 else 1e-6), f
    if prec == FP64:
        assert t == t_ref
        assert np.all(_rel(got[live], ref[live]) <= TOL_FP64), _rel(got[live], ref[live])
    else:
        assert t == pytest.approx(t_ref, rel=1e-5)
        err = l1rel(got[live].reshape(len(live), -1), ref[live].reshape(len(live), -1))
        assert np.all(err <= TOL_FP32_L1), err


def _oracle_run_to(oracle, pr, w, t_end):
    """CFL steps of the oracle until t_end, the last one clipped onto it."""
    t, n = 0.0, 0
    while t < t_end:
        cm = oracle.cmax3(pr, w)
        dt = oracle.cfl_dt3(pr, *cm)
        last = t + dt >= t_end
        if last:
            dt = t_end - t
        w = oracle.rk4_step3(pr, w, dt, cm)
        t = t_end if last else t + dt
        n += 1
    return w, n


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_run_to_lands_on_t_end(oracle_mod, inputs_mod, precision):
    from paper_1710_06423_b300.sac import FP32, FP64, Solver3
    prec = FP64 if precision == "fp64" else FP32
    nx, ny, nz = 18, 14, 10
    t_end = 0.0312
    w = inputs_mod.ot_3d(nx, ny, nz, compress=0.3)
    pr = oracle_mod.Problem3(nx=nx, ny=ny, nz=nz)
    ref, n_ref = _oracle_run_to(oracle_mod, pr, w, t_end)
    with Solver3(nx=nx, ny=ny, nz=nz, precision=prec) as s:
        s.set_state(w, 0.0)
        n = s.run_to(t_end)
        got, t = s.get_state()
        assert s.run_to(t_end) == 0            # already there: no further step
    assert t == t_end and n >= 2
    if prec == FP64:
        assert n == n_ref
        assert np.all(_rel(got, ref) <= TOL_FP64), _rel(got, ref)
    else:
        assert abs(n - n_ref) <= 1
        err = l1rel(got.reshape(8, -1), ref.reshape(8, -1))
        assert np.all(err <= TOL_FP32_L1), err
