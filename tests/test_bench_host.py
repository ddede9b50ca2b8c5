"""Host logic of bench.py's reference arm (no GPU): the oracle's timed
steps stop once their time budget is spent, and the band sample of a
graded set has every resolution of the set."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2107_01276_gb300 import workloads as wl  # noqa: E402


def test_oracle_steps_stop_at_the_budget():
    d = wl.taylor_green(nx=12)
    ps, el, threads, run = bench.oracle_steps(d, d["particles"], 5, False, budget_s=0.0)
    assert run == 1 and ps == len(d["particles"]["x"]) and el > 0 and threads >= 1
    ps, el, threads, run = bench.oracle_steps(d, d["particles"], 3, False)
    assert run == 3 and ps == 3 * len(d["particles"]["x"])


def test_band_sample_keeps_every_resolution():
    d = wl.graded_strip(n_target=40000, ratio=16.0)
    sd, n, frac = bench.cpu_sample(d, 0.05)
    assert frac == 0.05 and n == len(sd["particles"]["x"]) and 0 < n < len(d["particles"]["x"])
    # the band is non-periodic in y and holds the finest and the coarsest h
    assert sd["params"]["periodic"][1] == 0
    h_all, h_band = d["particles"]["h"], sd["particles"]["h"]
    assert np.isclose(h_band.min(), h_all.min()) and np.isclose(h_band.max(), h_all.max())
