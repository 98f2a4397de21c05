"""Host logic of the measurement script (no GPU): the learned-proposal statistics (first step within the
target tolerance, convergence test, the runs that miss the target), the traffic line lookup in the
committed ncu summaries, and the work models behind the roofline fractions."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_steps_to_target_first_step_within_tolerance():
    target = np.array([10.0, -5.0, 3.0])
    trace = np.array([[12.0, -4.0, 4.0],
                      [10.0 + 2e-5, -5.0 + 4e-6, 3.5],
                      [9.0, -6.0, 3.2]])
    # tolerance 1e-6 |target|: fit 0 reaches 10 only at step 2 (2e-5 above is outside 1e-5); fit 1 at step 1
    # (4e-6 <= 5e-6); fit 2 never
    assert list(bench.steps_to_target(trace, target)) == [2, 1, -1]


def test_converged_uses_running_best_over_the_window():
    # window 2: the running best at the last step against the one two steps earlier.  Fit 0 still improves
    # by 1e-3, fit 1 is flat, fit 2 is flat apart from a NaN step (ignored), fit 3 improved inside the window
    tr = np.array([[3.0, 2.0, 4.0, 6.0], [2.0, 2.0, np.nan, 5.0], [1.999, 2.0, 4.0, 4.0], [1.998, 2.0, 4.0, 4.0]])
    assert [bool(v) for v in bench.converged(tr, 2)] == [False, True, True, False]


def test_unreached_summary():
    target = np.array([1.0, 2.0, 4.0])
    prop = np.array([[3.0, 3.0, 5.0], [2.0, 2.5, 4.5], [1.5, 2.4, 4.4], [1.5, 2.2, 4.4]])
    reached = np.array([True, False, False])
    s = bench.unreached_summary(prop, target, reached, 1)
    assert s["fits"] == 2
    assert s["best_excess_median"] == pytest.approx(np.median([0.2 / 2.0, 0.4 / 4.0]))
    assert s["best_excess_max"] == pytest.approx(0.1)
    assert s["converged_fraction"] == pytest.approx(0.5)     # fit 2 flat over the last step, fit 1 not
    assert bench.unreached_summary(prop, target, np.ones(3, bool), 1) == {"fits": 0}


def test_profile_traffic_matches_current_sources_only():
    sha = bench.kernel_sources_sha()
    assert len(sha) == 16
    v = bench.profile_traffic("k_rt_b")
    assert v is None or v > 0
    assert bench.profile_traffic("no_such_kernel") is None


def test_work_models():
    # kernel B: double-float flops per frequency grow with T; the FP64-equivalent view is 120 flops at T = 4
    assert bench.df_solve_flops_per_freq(4, True) > bench.df_solve_flops_per_freq(4, False) > 0
    assert bench.df_solve_flops_per_freq(8, True) > bench.df_solve_flops_per_freq(4, True)
    assert bench.fp64_equivalent(65536, 4, 1e-3)["flops_per_frequency"] == pytest.approx(120.0)
    # kernels A and C: operations per item are affine in d and in the stages a
    a8, a9 = bench.rt_item_ops("a", 8, 8), bench.rt_item_ops("a", 8, 9)
    assert a9 - a8 == 1
    assert bench.rt_item_ops("a", 9, 8) - a8 == bench.rt_item_ops("a", 10, 8) - bench.rt_item_ops("a", 9, 8)
    assert bench.rt_item_ops("c", 8, 8) < a8
    # the posterior's double-float pair model
    assert bench.pd_pair_ops(8) == 8 * bench.PD_OPS_DIM + bench.PD_OPS_ACC
