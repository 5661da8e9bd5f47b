"""Bounded device waits.

The FP32 stage kernels wait on an mbarrier for their staging copies and give
up after about one second, recording a timeout in the run's status instead of
hanging the GPU.  These tests make that wait run out on purpose, the way the
test hook documented in sac.h does it: the stage kernels issue no copies, so
the expected bytes never arrive.  Nothing faults and no copy is left in
flight.  The step must report SAC_ERR_TIMEOUT within seconds, and the context
must stay usable: after the hook is cleared it reproduces an untouched run
bit for bit.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_2d_copy_wait_times_out_and_context_recovers(inputs_mod):
    from paper_1710_06423_b300.sac import FP32, SAC_ERR_TIMEOUT, SacError, Solver
    n = 96
    w = inputs_mod.orszag_tang(n, noise=1e-3, seed=5)
    with Solver(nx=n, ny=n, precision=FP32) as ref:
        ref.set_state(w, None, 0.0)
        ref.steps(2)
        want, t_want = ref.get_state()
    with Solver(nx=n, ny=n, precision=FP32) as s:
        s.set_state(w, None, 0.0)
        s.debug_drop_copies(True)
        t0 = time.perf_counter()
        with pytest.raises(SacError) as err:
            s.step()
        elapsed = time.perf_counter() - t0
        assert err.value.code == SAC_ERR_TIMEOUT
        assert elapsed < 30.0, elapsed
        # later steps are skipped until the state is set again
        with pytest.raises(SacError) as err2:
            s.step()
        assert err2.value.code == SAC_ERR_TIMEOUT
        s.debug_drop_copies(False)
        s.set_state(w, None, 0.0)
        s.steps(2)
        got, t = s.get_state()
    assert t == t_want
    assert np.array_equal(got, want)


def test_3d_copy_wait_times_out_and_context_recovers(inputs_mod):
    from paper_1710_06423_b300.sac import FP32, SAC_ERR_TIMEOUT, SacError, Solver3
    n = 24
    w = inputs_mod.ot_3d(n, n, n, compress=0.3)
    with Solver3(nx=n, ny=n, nz=n, precision=FP32) as ref:
        ref.set_state(w, 0.0)
        start, _ = ref.get_state()
        ref.steps(2)
        want, t_want = ref.get_state()
    with Solver3(nx=n, ny=n, nz=n, precision=FP32) as s:
        s.set_state(w, 0.0)
        s.debug_drop_copies(True)
        t0 = time.perf_counter()
        with pytest.raises(SacError) as err:
            s.step()
        elapsed = time.perf_counter() - t0
        assert err.value.code == SAC_ERR_TIMEOUT
        assert elapsed < 30.0, elapsed
        kept, t_kept = s.get_state()            # the abandoned step left the state as it was
        assert t_kept == 0.0 and np.array_equal(kept, start)
        s.debug_drop_copies(False)
        s.steps(2)
        got, t = s.get_state()
    assert t == t_want
    assert np.array_equal(got, want)


def test_hooks_reject_fp64_contexts():
    from paper_1710_06423_b300.sac import FP64, SAC_ERR_ARG, SacError, Solver, Solver3
    with Solver(nx=16, ny=16, precision=FP64) as s:
        with pytest.raises(SacError) as err:
            s.debug_drop_copies(True)
        assert err.value.code == SAC_ERR_ARG
    with Solver3(nx=8, ny=8, nz=8, precision=FP64) as s3:
        with pytest.raises(SacError) as err:
            s3.debug_drop_copies(True)
        assert err.value.code == SAC_ERR_ARG
