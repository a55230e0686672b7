"""Step-size balancing and the cost function (oracle, test infrastructure).

* ``balance_steps`` (Sec. 2.4, eq. force_tune): step sizes with F_i h_i = constant, F_i
  the maximal force of level i (the paper balances the maximal forces).  Anchored at the
  level with the smallest force, which keeps n_coarse steps over tau; every other level
  gets n_i = n_coarse F_i / F_coarse steps, rounded to the nearest integer (at least
  one), since a level must take a whole number of steps over tau.
* ``cost`` (Sec. 3.1, eqs. cost_func and error_corrected): over N trajectories,
  P_acc = mean(accepted), N_mat = mean(K/J applications), C = N_mat / P_acc, each error
  sigma = sqrt(2 tau_int) sigma_p / sqrt(N) with sigma_p the sample standard deviation
  (N - 1 in the denominator); the error of C follows from those of N_mat and P_acc by
  linear propagation (the paper gives no formula for it); <exp(-dH)> with the same error.
"""
import math


def balance_steps(fmax, n_coarse):
    c = min(range(len(fmax)), key=lambda i: fmax[i])
    return [max(1, int(math.floor(n_coarse * f / fmax[c] + 0.5))) for f in fmax]


def _mean_err(xs, tau_int):
    n = len(xs)
    m = sum(xs) / n
    if n < 2:
        return m, float("nan")
    sp = math.sqrt(sum((x - m) ** 2 for x in xs) / (n - 1))
    return m, math.sqrt(2.0 * tau_int) * sp / math.sqrt(n)


def cost(accepted, nmat, dH, tau_int=12.5):
    p, ep = _mean_err([1.0 if a else 0.0 for a in accepted], tau_int)
    nm, en = _mean_err(list(nmat), tau_int)
    ex, ee = _mean_err([math.exp(-d) for d in dH], tau_int)
    c = nm / p if p > 0 else float("inf")
    ec = c * math.sqrt((en / nm) ** 2 + (ep / p) ** 2) if p > 0 else float("inf")
    return {"p_acc": p, "p_acc_err": ep, "nmat": nm, "nmat_err": en, "cost": c, "cost_err": ec,
            "exp_mdh": ex, "exp_mdh_err": ee}
