"""Pins of the oracle's step balancing (Sec. 2.4) and cost function (Sec. 3.1) against
values worked out by hand."""
import math

from oracle.tuning import balance_steps, cost


def test_balance_steps_force_times_step_constant():
    # forces 0.5, 1.0, 2.5, 7.5 with 4 steps on the weakest level: 4, 8, 20, 60 steps,
    # so that F_i h_i = F_i tau / n_i = 0.125 tau on every level
    n = balance_steps([0.5, 1.0, 2.5, 7.5], 4)
    assert n == [4, 8, 20, 60]
    assert len({f / k for f, k in zip([0.5, 1.0, 2.5, 7.5], n)}) == 1
    # the anchor is the smallest force wherever it sits; rounding to the nearest integer
    assert balance_steps([3.0, 1.0, 1.6], 5) == [15, 5, 8]
    assert balance_steps([1.0, 1.0], 3) == [3, 3]


def test_cost_hand_example():
    """accepted 1,1,0,1: P_acc = 3/4, sample variance 1/4, sigma = sqrt(25) (1/2) / 2 = 1.25;
    N_mat 100,120,80,100: mean 100, sample variance 800/3, sigma = 5 sqrt(800/3) / 2."""
    r = cost([1, 1, 0, 1], [100, 120, 80, 100], [0.1, -0.2, 1.5, 0.0], tau_int=12.5)
    assert abs(r["p_acc"] - 0.75) < 1e-15
    assert abs(r["p_acc_err"] - 1.25) < 1e-14
    assert abs(r["nmat"] - 100.0) < 1e-12
    en = 2.5 * math.sqrt(800.0 / 3.0)
    assert abs(r["nmat_err"] - en) < 1e-11
    assert abs(r["cost"] - 400.0 / 3.0) < 1e-12
    assert abs(r["cost_err"] - (400.0 / 3.0) * math.sqrt((en / 100) ** 2 + (1.25 / 0.75) ** 2)) < 1e-9
    ex = (math.exp(-0.1) + math.exp(0.2) + math.exp(-1.5) + 1.0) / 4
    assert abs(r["exp_mdh"] - ex) < 1e-15
