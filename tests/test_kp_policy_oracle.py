"""Pins for the reference of the learned budget-level choice
(oracle/kp_policy.py), worked by hand from its definition: level l keeps
ceil(P / 2^shift) postings, needs k' = max(ceil(2^(y + margin)), kp_min),
is feasible when that is at most kp_max, and the feasible level of least
posting_cost * postings + k' wins (ties: the earlier level); with none
feasible, the whole query at kp_max."""
import numpy as np

from oracle import kp_policy


def test_level_budgets():
    assert kp_policy.level_budget(100000, 0) == 0          # the whole query: no break
    assert kp_policy.level_budget(100000, 1) == 50000
    assert kp_policy.level_budget(100001, 1) == 50001      # rounded up
    assert kp_policy.level_budget(7, 3) == 1
    assert kp_policy.level_budget(0, 4) == 0
    assert kp_policy.level_postings(12345, 0) == 12345


def test_hand_worked_choices():
    shifts = (0, 1, 2)
    P = np.array([100000, 50000, 80000, 40000])
    y = np.array([
        [5.0, 6.0, 13.0],    # k' 32, 64, 8192 (infeasible): costs 132, 114 -> level 1
        [3.0, 3.0, 3.0],     # k' 8 -> kp_min 10: costs 60, 35, 22.5 -> level 2
        [20.0, 20.0, 20.0],  # nothing feasible -> level 0 at kp_max
        [4.0, 5.0, 2.0],     # k' 16, 32, 10: costs 56, 52, 20 -> level 2
    ], np.float32)
    kp, bud, lev, cost = kp_policy.choose(y, P, shifts, 0.001, 0.0, 10, 4096)
    assert list(lev) == [1, 2, 0, 2]
    assert list(kp) == [64, 10, 4096, 10]
    assert list(bud) == [50000, 12500, 0, 10000]
    assert abs(cost[0, 0] - 132.0) < 1e-4 and abs(cost[0, 1] - 114.0) < 1e-4
    assert np.isinf(cost[0, 2]) and np.isinf(cost[2]).all()
    assert abs(cost[1, 2] - 22.5) < 1e-4


def test_margin_ceil_and_ties():
    # margin 1 doubles every k': 2^(5+1) = 64 and 2^(6+1) = 128, costs
    # 100 + 64 = 164 and 50 + 128 = 178 -> level 0; without the margin the
    # costs are 132 and 114 -> level 1
    kp, bud, lev, _ = kp_policy.choose(np.array([[5.0, 6.0]], np.float32), np.array([100000]),
                                       (0, 1), 0.001, 1.0, 10, 4096)
    assert list(lev) == [0] and list(kp) == [64] and list(bud) == [0]
    kp, bud, lev, _ = kp_policy.choose(np.array([[5.0, 6.0]], np.float32), np.array([100000]),
                                       (0, 1), 0.001, 0.0, 10, 4096)
    assert list(lev) == [1] and list(kp) == [64] and list(bud) == [50000]
    # 2^5.5 = 45.25 -> 46
    kp, _, _, _ = kp_policy.choose(np.array([[5.5]], np.float32), np.array([10]), (0,), 0.0, 0.0,
                                   10, 4096)
    assert list(kp) == [46]
    # equal costs: 0 postings cost, k' 32 on both levels -> the earlier level
    kp, bud, lev, _ = kp_policy.choose(np.array([[5.0, 5.0]], np.float32), np.array([1000]),
                                       (0, 3), 0.0, 0.0, 10, 4096)
    assert list(lev) == [0] and list(bud) == [0]
    # negative outputs clamp to 2^0 = 1 -> kp_min
    kp, _, _, _ = kp_policy.choose(np.array([[-3.0]], np.float32), np.array([1]), (0,), 0.0, 0.0,
                                   10, 4096)
    assert list(kp) == [10]
    # exactly at the cap is feasible, one above is not
    kp, _, lev, _ = kp_policy.choose(np.array([[12.0, 12.01]], np.float32), np.array([4096]),
                                     (0, 1), 1.0, 0.0, 10, 4096)
    assert list(lev) == [0] and list(kp) == [4096]
