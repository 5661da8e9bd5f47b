"""How much the Brio-Wu shock tube itself amplifies a rounding-sized change of
its state (FP64 oracle only, no GPU).

This is the measurement behind the FP32 Brio-Wu tolerance of the GPU tests
(1e-3 relative L1 per field instead of the smooth-flow 1e-5): two FP64 oracle
runs to t = 0.1 whose starts differ by a relative 2^-24 (one FP32 rounding of
each value) end 1e-4 .. 1e-3 apart in the momenta, because the shocks turn a
change of the state into a shift of their positions.  A single-precision run,
which rounds at every stage of about 1040 steps, cannot be closer to the
oracle than the oracle is to itself under such a change.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.slow


def test_brio_wu_amplifies_a_single_fp32_rounding(oracle_mod, inputs_mod):
    pr = oracle_mod.Problem(nx=800, ny=1, gamma=2.0, bc_x=1)
    w0 = inputs_mod.brio_wu()
    ref, t, n = oracle_mod.run(pr, w0, t_end=0.1)
    rng = np.random.default_rng(0)
    w1 = w0 * (1.0 + 2.0 ** -24 * rng.uniform(-1.0, 1.0, w0.shape))
    got, t1, n1 = oracle_mod.run(pr, w1, t_end=0.1)
    assert t == t1 == 0.1 and n == n1
    num = np.abs(got - ref).reshape(6, -1).sum(1)
    den = np.abs(ref).reshape(6, -1).sum(1)
    err = num / den
    # momentum: 4e-4 measured (three seeds: 4.2e-4 .. 4.9e-4)
    assert 1e-4 <= err[1] <= 1e-3, err
    # every field but the exactly conserved B_x moves by far more than 1e-5
    assert np.all(err[[0, 1, 2, 3, 5]] > 1e-5), err
    assert err[4] < 1e-7, err
