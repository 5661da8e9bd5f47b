"""Host logic of the learned-correction experiment (no GPU): the equal-error
interpolation, the m-step pair targets and the bookkeeping of pair sets."""
import math

import numpy as np
import pytest


def test_equal_error_time_is_log_log_interpolation():
    from paper_1710_06423_b300.learned import equal_error_time
    # error proportional to 1/time: the point at error 0.05 lies at time 2
    curve = [(4.0, 0.025), (1.0, 0.1), (16.0, 0.00625)]
    assert math.isclose(equal_error_time(curve, 0.05), 2.0, rel_tol=1e-12)
    assert math.isclose(equal_error_time(curve, 0.0125), 8.0, rel_tol=1e-12)
    assert equal_error_time(curve, 0.2) is None          # worse than the coarsest plain run
    assert equal_error_time(curve, 0.001) is None        # better than the finest


def test_pair_targets_share_and_whole():
    import torch
    from paper_1710_06423_b300.learned import Pairs, _target
    rng = np.random.default_rng(3)
    xp = torch.from_numpy(rng.standard_normal((6, 5, 5)).astype(np.float32))
    raw = torch.from_numpy(rng.standard_normal((6, 5, 5)).astype(np.float32))
    share, whole, one = Pairs(4, share=True), Pairs(4, share=False), Pairs(1)
    assert (share.apply_every, whole.apply_every, one.apply_every) == (1, 4, 1)
    got = _target(share, xp, raw, torch)
    assert torch.allclose(got.double(), xp.double() + (raw.double() - xp.double()) / 4, atol=1e-6)
    assert _target(whole, xp, raw, torch) is raw
    assert _target(one, xp, raw, torch) is raw


def test_select_and_merge_keep_pair_kind():
    from paper_1710_06423_b300.learned import Pairs, merged, select
    a, b = Pairs(8, share=False), Pairs(8, share=False)
    for k in range(3):
        a.x.append(k); a.next.append(10 + k); a.raw.append(20 + k); a.gamma.append(1.4); a.meta.append((0, 8 * k))
    b.x.append(9); b.next.append(19); b.raw.append(29); b.gamma.append(5 / 3); b.meta.append((1, 0))
    a.final[0] = "fine0"
    b.final[1] = "fine1"
    s = select(a, np.array([True, False, True]))
    assert (s.substeps, s.share, s.apply_every) == (8, False, 8)
    assert s.x == [0, 2] and s.next == [10, 12] and s.raw == [20, 22] and s.meta == [(0, 0), (0, 16)]
    m = merged(a, b)
    assert len(m) == 4 and m.raw[-1] == 29 and m.final == {0: "fine0", 1: "fine1"}
    assert (m.substeps, m.share) == (8, False)


def test_generate_pairs_rejects_windows_longer_than_the_spacing():
    import torch
    from paper_1710_06423_b300 import learned
    with pytest.raises(ValueError):
        learned.generate_pairs(learned.Pairs(16), 1, 0, 32, 4, 1e-3, n_steps=60, every=15, torch=torch)
