"""Host-side pieces of bench.py: the algorithmic work count behind the roofline
fraction (node counts per band against the oracle's rules) and the clock
sampler's timed-window filter."""
import numpy as np

import bench
import oracle


def test_algorithmic_work_counts_the_rule_of_each_band():
    """Bands 1..5 are the 33, 19|17, 12, 7 and 4-point rules (band 0 is the
    analytic near field, no cubature work): 8 + 13 N operations and N rsqrt
    per pair, with N the size of the oracle's rule."""
    rng = np.random.default_rng(0)
    stats = rng.integers(0, 1000, size=12).astype(float)
    ops, rsq, flops = bench.algorithmic_work(stats)
    e_ops = e_rsq = e_flops = 0.0
    for t in (0, 1):
        for band in range(1, 6):
            n = oracle.rule(t, 5 - band).shape[0]  # rule index 4 = 33 points ... 0 = 4 points
            e_ops += stats[6 * t + band] * (8 + 13 * n)
            e_flops += stats[6 * t + band] * (8 + 18 * n)
            e_rsq += stats[6 * t + band] * n
    assert (ops, rsq, flops) == (e_ops, e_rsq, e_flops)
    # near pairs cost nothing here
    only_near = np.zeros(12)
    only_near[[0, 6]] = 5.0
    assert bench.algorithmic_work(only_near) == (0.0, 0.0, 0.0)


def test_clock_sampler_keeps_the_timed_window():
    cs = bench.ClockSampler(0)
    row = ["2070", "2070", "500", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    slow = ["1200", "2070", "500", "0x0", "Not Active", "Not Active", "Not Active", "Active"]
    cs.rows = [(0.0, slow), (1.0, row), (1.5, row), (3.0, slow)]
    cs.t0, cs.t1 = 0.9, 2.0
    out = cs.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == 2070.0 and out["reasons"] == []
    # a window shorter than one sampling period keeps every sample
    cs = bench.ClockSampler(0)
    cs.rows = [(0.0, slow), (1.0, row)]
    cs.t0, cs.t1 = 5.0, 5.1
    out = cs.stop()
    assert out["samples"] == 2 and out["reasons"] == ["sw_power_cap"]
