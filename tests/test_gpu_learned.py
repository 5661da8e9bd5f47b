"""The learned coarse-grid correction end to end at a small scale: training data
from the fine solver, training on the GPU with the project's kernels, and what
the trained network gains over the plain coarse method on held-out runs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import torch
    from paper_1710_06423_b300 import learned
    from paper_1710_06423_b300.sac import CNN
    nc, ratio = 32, 4
    dx = 1.0 / nc
    dt_c = 0.2 * dx / 2.5
    pairs = learned.Pairs()
    for k in range(3):
        learned.generate_pairs(pairs, 77, k, nc, ratio, dt_c, n_steps=60, every=3, torch=torch)
    held = learned.Pairs()
    learned.generate_pairs(held, 77, 10, nc, ratio, dt_c, n_steps=60, every=3, torch=torch)
    osc = learned.out_scales(pairs, torch)
    net = CNN(nc, nc)
    net.set_params(learned.init_params(1))
    net.set_scales(learned.FEATURE_SCALES, osc)
    untrained_gain = learned.residual_gain(net, held, osc, dx, torch)
    losses = learned.train(net, pairs, osc, dx, iters=600, lr=2e-3, torch=torch, log_every=100)
    return dict(net=net, pairs=pairs, held=held, osc=osc, dx=dx, dt_c=dt_c, nc=nc, ratio=ratio,
                untrained_gain=untrained_gain, losses=losses)


def test_training_loss_falls(trained):
    losses = trained["losses"]
    assert losses[-1][1] < 0.7 * losses[0][1], losses


def test_trained_network_reduces_one_step_residual_on_held_out_run(trained):
    import torch
    from paper_1710_06423_b300 import learned
    gain = learned.residual_gain(trained["net"], trained["held"], trained["osc"], trained["dx"], torch)
    # 1.0 = the plain coarse step; the untrained network starts near 1
    assert gain < 0.85 and gain < trained["untrained_gain"] - 0.1, (gain, trained["untrained_gain"])


def test_learned_rollout_beats_plain_coarse(trained):
    """Held-out family member: 60 coarse steps with and without the correction,
    compared with the block-averaged fine run at the same time."""
    import torch
    from paper_1710_06423_b300 import learned
    from paper_1710_06423_b300.sac import FP32, Solver, block_average
    nc, ratio, dt_c = trained["nc"], trained["ratio"], trained["dt_c"]
    nf = nc * ratio
    w0f, gamma = learned.family_state(77, 11, nf)
    steps = 60
    fine_out = torch.empty((6, nf, nf), dtype=torch.float32, device="cuda")
    with Solver(nx=nf, ny=nf, precision=FP32, gamma=gamma) as fine:
        fine.set_state(w0f, None, 0.0)
        fine.set_fixed_dt(dt_c / ratio)
        fine.steps(steps * ratio)
        fine.get_state_dev(fine_out)
    truth = torch.empty((6, nc, nc), dtype=torch.float32, device="cuda")
    block_average(fine_out, 6, nf, nf, ratio, truth)
    w0c = torch.empty_like(truth)
    block_average(torch.from_numpy(w0f.astype(np.float32)).cuda().contiguous(), 6, nf, nf, ratio, w0c)
    w0c = w0c.double().cpu().numpy()
    plain, _ = learned.run_plain(w0c, gamma, nc, dt_c, steps, torch)
    corr, _ = learned.run_plain(w0c, gamma, nc, dt_c, steps, torch, net=trained["net"])
    e_plain = learned.l1_error(plain, truth)
    e_corr = learned.l1_error(corr, truth)
    assert e_corr.mean() < e_plain.mean(), (e_corr, e_plain)


def test_multi_step_pairs():
    """Pairs over m = 4 coarse steps: one pair every 6 steps over 24 steps, the
    coarse input is 4 plain steps from the block-averaged fine state, and the
    target is the per-step share x' + (avg fine(t + 4 dt) - x') / 4; the final
    block-averaged fine state is kept for the member."""
    import torch
    from paper_1710_06423_b300 import learned
    from paper_1710_06423_b300.sac import FP32, Solver, block_average
    nc, ratio = 32, 4
    dt_c = 0.2 / nc / 2.5
    pairs = learned.Pairs(4)
    done = learned.generate_pairs(pairs, 77, 0, nc, ratio, dt_c, n_steps=24, every=6, torch=torch)
    assert done == 24 and len(pairs) == 4 and [m for _, m in pairs.meta] == [0, 6, 12, 18]
    assert 0 in pairs.final
    for xp, nxt, raw in zip(pairs.x, pairs.next, pairs.raw):
        want = xp.double() + (raw.double() - xp.double()) / 4
        assert torch.allclose(nxt.double(), want, rtol=1e-6, atol=1e-7)
    # the second pair's input: 4 plain coarse steps from avg(fine) at coarse step 6
    nf = nc * ratio
    w0f, gamma = learned.family_state(77, 0, nf)
    fine_buf = torch.empty((6, nf, nf), dtype=torch.float32, device="cuda")
    a0 = torch.empty((6, nc, nc), dtype=torch.float32, device="cuda")
    xp = torch.empty_like(a0)
    with Solver(nx=nf, ny=nf, precision=FP32, gamma=gamma) as fine, \
            Solver(nx=nc, ny=nc, precision=FP32, gamma=gamma) as coarse:
        fine.set_state(w0f, None, 0.0)
        fine.set_fixed_dt(dt_c / ratio)
        fine.steps(6 * ratio)
        fine.get_state_dev(fine_buf)
        block_average(fine_buf, 6, nf, nf, ratio, a0)
        coarse.set_state_dev(a0, None, 0.0)
        for _ in range(4):
            coarse.step(dt_c)
        coarse.get_state_dev(xp)
        coarse.sync()
    assert torch.equal(xp, pairs.x[1])
