"""Numbers the paper prints, kept as text fixtures under tests/golden/ (each
with its passage), against what the code builds from them:

* the Brio-Wu left/right states (section 5.2) against the initial state the
  input generator produces (primitive values recovered from the conserved
  fields on each side of the discontinuity);
* the Orszag-Tang timings of Table 1 (section 5.1) against the paper rate the
  benchmark divides by (8000^2 with hyper-diffusion on 10 x 10 GPUs, 100
  iterations).
"""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_brio_wu_states_match_the_paper(inputs_mod):
    states = {r[0]: (float(r[1]), float(r[2])) for r in _rows("brio_wu_states.txt")}
    gamma = 2.0
    n = 800
    w = inputs_mod.brio_wu(n, 1, gamma=gamma)
    rho, mx, my, e, bx, by = (a[0] for a in w)
    x = (np.arange(n) + 0.5) / n
    for side, sel in ((0, x < 0.5), (1, x > 0.5)):
        r = rho[sel]
        vx, vy = mx[sel] / r, my[sel] / r
        p = (gamma - 1.0) * (e[sel] - 0.5 * r * (vx * vx + vy * vy) - 0.5 * (bx[sel] ** 2 + by[sel] ** 2))
        np.testing.assert_allclose(r, states["rho"][side], rtol=0, atol=1e-15)
        np.testing.assert_allclose(p, states["p"][side], rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(by[sel], states["By"][side], rtol=0, atol=0)
        np.testing.assert_allclose(bx[sel], states["Bx"][side], rtol=0, atol=0)
        assert np.all(vx == 0.0) and np.all(vy == 0.0)


def test_table1_rate_used_by_the_benchmark():
    rows = _rows("table1_timings.txt")
    hd = {(int(r[0]), r[1]): float(r[3]) for r in rows if r[3] != "-"}
    assert len(rows) == 8 and len(hd) == 5
    # time with hyper-diffusion always exceeds the time without it
    for r in rows:
        if r[3] != "-":
            assert float(r[3]) > float(r[2])
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(os.path.dirname(HERE), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    rate = 8000 * 8000 * 100 / hd[(8000, "10x10")]
    assert bench.PAPER_8000_HD == pytest.approx(rate, rel=1e-12)
    assert rate == pytest.approx(3.91e7, rel=2e-3)
