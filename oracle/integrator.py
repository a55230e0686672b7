"""MD integrators and the HMC trajectory of the oracle (test infrastructure).

* Step arrays (App. B, "Example algorithm"): a scheme is a pair of arrays T, S enacted as
  ``for i: T-hat[T[i]]; S-hat[S[i]]``.
* 2MN (eq. 2MNSTS): S[lam h] T[h/2] S[(1 - 2 lam) h] T[h/2] S[lam h], n steps chained, the
  touching S[lam h] S[lam h] of neighbouring steps combined (S-hat[a+b] = S-hat[a] S-hat[b]).
* Leapfrog: S[h/2] T[h] S[h/2] per step.
* ``merge``: the generalised multi-scale integrator (eq. uber_gen) built by the merge
  procedure of App. B: repeatedly take the smallest pending time step, emit it, emit the
  S step of every scheme whose pending time step it completes (0 for the others) and
  shorten the others' pending time steps.  The paper compares the pending time steps
  with ``==``; on floating-point step sizes that is read as equality within ``eps``.
* ``trajectory``: H = sum tr P^2 + S (Sec. 2.1), T-hat: U -> exp(i eps P) U, S-hat:
  P -> P - eps F, Metropolis accept iff u < exp(-(H' - H)).
"""
import math

import torch

from .lattice import algebra_to_matrix, expi_hermitian

LAMBDA_2MN = 0.1931833275037836


def two_mn(n, tau, lam=LAMBDA_2MN):
    h = tau / n
    T = [0.0] + [h / 2] * (2 * n)
    S = [lam * h]
    for k in range(n):
        S.append((1 - 2 * lam) * h)
        S.append(2 * lam * h if k < n - 1 else lam * h)
    return T, S


def leapfrog(n, tau):
    h = tau / n
    return [0.0] + [h] * n, [h / 2] + [h] * (n - 1) + [h / 2]


def merge(schemes, eps=1e-12):
    """Merge per-term (T, S) arrays into (T', [S'_1, S'_2, ...]) (App. B)."""
    Ts = [list(T) for T, _ in schemes]
    Ss = [list(S) for _, S in schemes]
    newT, newS = [], [[] for _ in schemes]
    while any(Ts):
        d = min(T[0] for T in Ts if T)
        newT.append(d)
        for i, T in enumerate(Ts):
            if T and abs(T[0] - d) <= eps:
                newS[i].append(Ss[i].pop(0))
                T.pop(0)
            else:
                newS[i].append(0.0)
                if T:
                    T[0] -= d
    return newT, newS


def kinetic(p):
    """sum_x,mu tr P^2 with P = sum_a p_a T_a: tr P^2 = (1/2) sum_a p_a^2."""
    return 0.5 * (p * p).sum().item()


def link_update(U, p, eps):
    return expi_hermitian(algebra_to_matrix(p), eps) @ U


def trajectory(action, U0, p0, xis, u, levels, schedule):
    """One PF-MP trajectory.

    action   oracle.action.PFMP
    levels   list of lists of term names per scheme, term names in
             {"gauge", "det", "poly", "polycorr", "hasen"}
    schedule merged (T', [S'_j]) from ``merge``
    Returns a dict with H0, H1, dH, accepted, U (the new field) and the trajectory end
    state before the accept/reject (U1, p1).
    """
    phi1, phi2, phi3 = action.heatbath(U0, *xis)

    def total_S(U):
        s = {}
        s["gauge"] = action.S_gauge(U).item()
        s["det"] = action.S_det(U).item() if action.p.csw != 0 else 0.0
        s["poly"] = action.S_poly(U, phi1).item()
        s["polycorr"] = action.S_polycorr(U, phi2).item()
        s["hasen"] = action.S_hasen(U, phi3).item()
        return s

    def force(name, U):
        if name == "gauge":
            return action.F_gauge(U)
        if name == "det":
            return action.F_det(U)
        if name == "poly":
            return action.F_poly(U, phi1)
        if name == "polycorr":
            return action.F_polycorr(U, phi2)
        if name == "hasen":
            return action.F_hasen(U, phi3)
        raise ValueError(name)

    S0 = total_S(U0)
    H0 = kinetic(p0) + sum(S0.values())
    U, p = U0.clone(), p0.clone()
    T, Slev = schedule
    for i in range(len(T)):
        if T[i] != 0.0:
            U = link_update(U, p, T[i])
        for j, names in enumerate(levels):
            eps = Slev[j][i]
            if eps != 0.0:
                for name in names:
                    p = p - eps * force(name, U)
    S1 = total_S(U)
    H1 = kinetic(p) + sum(S1.values())
    dH = H1 - H0
    accepted = bool(u < math.exp(-dH)) if dH > -700 else True
    return {
        "H0": H0, "H1": H1, "dH": dH, "accepted": accepted, "S0": S0, "S1": S1,
        "U1": U, "p1": p, "U": U if accepted else U0, "phi": (phi1, phi2, phi3),
    }


def trajectory_terms(action, U0, p0, xis, u, term_level, schedule):
    """One trajectory of a general ``oracle.action.Action``: term i is integrated on
    scheme ``term_level[i]`` of the merged schedule (-1: left out of H and of the MD)."""
    phis = action.heatbath(U0, xis)
    phi_of = {i: phis[k] for k, i in enumerate(action.pf)}
    used = [i for i, l in enumerate(term_level) if l >= 0]

    def total_S(U):
        return {i: action.S(U, i, phi_of.get(i)).item() for i in used}

    S0 = total_S(U0)
    H0 = kinetic(p0) + sum(S0.values())
    U, p = U0.clone(), p0.clone()
    T, Slev = schedule
    for k in range(len(T)):
        if T[k] != 0.0:
            U = link_update(U, p, T[k])
        for j in range(len(Slev)):
            eps = Slev[j][k]
            if eps != 0.0:
                for i in used:
                    if term_level[i] == j:
                        p = p - eps * action.F(U, i, phi_of.get(i))
    S1 = total_S(U)
    H1 = kinetic(p) + sum(S1.values())
    dH = H1 - H0
    accepted = bool(u < math.exp(-dH)) if dH > -700 else True
    return {
        "H0": H0, "H1": H1, "dH": dH, "accepted": accepted, "S0": S0, "S1": S1,
        "U1": U, "p1": p, "U": U if accepted else U0, "phi": phis,
    }
