"""GPU parity of the general actions (Sec. 2.2, 2.3, 2.5, 3.6) against the oracle at
4^4 (FP64): the scheme term lists, each fermion term's heatbath, action and force for
the factorised filter Q(J), the inverse and a Hasenbusch ratio between two
preconditioning kappas, and one trajectory each of 2PF-1MP and 1PF-2MP (Delta H within
1e-8 of the oracle's)."""
import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, canon, from_canon, oracle_gauge, rel_l2

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
KAPPAS = [0.120, 0.100, 0.110]
BETA, CSW, MU, NU, TOL = 5.5, 1.0, 1.2, 0.9, 1e-12

SCHEMES = {  # name: (C id, p1, p2, oracle kwargs)
    "1PF": (0, 0, 8, dict(p2=8)), "2PF": (1, 2, 8, dict(p1=2, p2=8)), "1MP": (2, 0, 0, {}), "2MP": (3, 0, 0, {}),
    "PF-MP": (4, 0, 8, dict(p2=8)), "2PF-1MP": (5, 2, 8, dict(p1=2, p2=8)), "1PF-2MP": (6, 0, 4, dict(p2=4)),
}
KIND = {"gauge": 0, "det": 1, "filter": 2, "filtercorr": 3, "ratio": 4, "inv": 5}


def _def(capi, scheme=None, terms=None):
    d = capi.ActionDef()
    d.beta, d.csw, d.nkappa = BETA, CSW, len(KAPPAS)
    for i, k in enumerate(KAPPAS):
        d.kappa[i] = k
    d.mu, d.nu, d.tol, d.max_iter = MU, NU, TOL, 5000
    if scheme is not None:
        cid, p1, p2, _ = SCHEMES[scheme]
        capi.pfmp_action_scheme(cid, p1, p2, d)
    else:
        d.nterms = len(terms)
        for i, t in enumerate(terms):
            d.term[i] = capi.Term(KIND[t.kind], t.a, t.b, t.p1, t.p2)
    return d


@pytest.fixture(scope="module")
def world():
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    yield lat, U, g, capi
    g.close()


def test_invalid_definitions(world):
    from oracle.action import Term

    lat, U, g, capi = world
    for terms in ([Term("filter", a=1, p1=4, p2=12)], [Term("filter", a=1, p2=7)], [Term("ratio", a=1, b=5)],
                  [Term("inv", a=4)]):
        with pytest.raises(capi.PfmpError):
            capi.pfmp_action_create_def(g.ctx, _def(capi, terms=terms))


def _noise(lat, n, base):
    return [lat.even * torch.tensor(pin.spinor(DIMS, base + k)).reshape(*lat.shape, 4, 3) for k in range(n)]


@pytest.mark.parametrize("name", ["2PF-1MP", "1PF-2MP", "2MP", "2PF"])
def test_heatbath_and_action_terms(world, name):
    from oracle.action import Action, scheme

    lat, U, g, capi = world
    act = Action(lat, BETA, CSW, KAPPAS, scheme(name, **SCHEMES[name][3]), mu=MU, nu=NU, tol=TOL)
    A = capi.pfmp_action_create_def(g.ctx, _def(capi, scheme=name))
    try:
        nt, npf = capi.pfmp_action_counts(A)
        assert (nt, npf) == (len(act.terms), len(act.pf))
        xi = _noise(lat, npf, 50)
        phis = act.heatbath(U, xi)
        capi.pfmp_action_heatbath(A, np.concatenate([canon(x) for x in xi]))
        for k in range(npf):
            out = np.zeros(lat.V * 24)
            capi.pfmp_action_get_phi(A, k, out)
            assert rel_l2(lat.even * from_canon(out, lat, (4, 3)), phis[k]) < 1e-10
        S = capi.pfmp_action_eval(A)
        for i in range(nt):
            phi = phis[act.pf.index(i)] if i in act.pf else None
            ref = act.S(U, i, phi).item()
            assert abs(S[i] - ref) < 1e-9 * max(1.0, abs(ref)), (name, i, S[i], ref)
        for k, i in enumerate(act.pf):     # heatbath identity
            assert abs(S[i] - (xi[k].abs() ** 2).sum().item()) < 1e-9 * S[i]
    finally:
        capi.pfmp_action_destroy(A)


@pytest.mark.parametrize("kind,a,b,p1,p2,tol", [("filter", 1, 0, 2, 8, 1e-11), ("filter", 0, 0, 4, 14, 1e-11),
                                               ("inv", 1, 0, 0, 0, 1e-9), ("ratio", 1, 2, 0, 0, 1e-9),
                                               ("filtercorr", 2, 0, 0, 4, 1e-9), ("det", 2, 0, 0, 0, 1e-11)],
                         ids=["Q(J)", "Q(K)", "inv", "ratio12", "filtercorr", "det"])
def test_force_terms(world, kind, a, b, p1, p2, tol):
    from oracle.action import Action, Term

    lat, U, g, capi = world
    t = Term(kind, a=a, b=b, p1=p1, p2=p2)
    act = Action(lat, BETA, CSW, KAPPAS, [t], mu=MU, nu=NU, tol=TOL)
    A = capi.pfmp_action_create_def(g.ctx, _def(capi, terms=[t]))
    try:
        phi = lat.even * torch.tensor(pin.spinor(DIMS, 61)).reshape(*lat.shape, 4, 3)
        if act.pf:
            capi.pfmp_action_set_phi(A, 0, canon(phi))
        F = np.zeros(lat.V * 32)
        capi.pfmp_action_force(A, 0, F)
        ref = act.F(U, 0, phi if act.pf else None)
        assert rel_l2(torch.tensor(F).reshape(*lat.shape, 4, 8), ref) < tol
    finally:
        capi.pfmp_action_destroy(A)


@pytest.mark.slow
@pytest.mark.parametrize("name,levels", [("2PF-1MP", [2, 2, 2, 1, 0, 0]), ("1PF-2MP", [2, 2, 2, 1, 0, 0])])
def test_trajectory_matches_oracle(name, levels):
    """Three-level 2MN (4, 8, 16 steps, tau = 0.5) with the gauge, determinant and first
    filter on the finest level: Delta H, H0 and the new field match the oracle."""
    from oracle.action import Action, scheme
    from oracle.integrator import LAMBDA_2MN, merge, trajectory_terms, two_mn
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    act = Action(lat, BETA, CSW, KAPPAS, scheme(name, **SCHEMES[name][3]), mu=MU, nu=NU, tol=TOL)
    xi = _noise(lat, len(act.pf), 70)
    p0 = torch.tensor(pin.momenta(DIMS, 8)).reshape(*lat.shape, 4, 8)
    u = float(pin.uniform(9)[0])
    tau = 0.5
    sched = merge([two_mn(4, tau), two_mn(8, tau), two_mn(16, tau)])
    ref = trajectory_terms(act, U, p0, xi, u, levels, sched)

    g = Gpu(lat, U)
    A = capi.pfmp_action_create_def(g.ctx, _def(capi, scheme=name))
    try:
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(n, tau, LAMBDA_2MN) for n in (4, 8, 16)])
        info = capi.pfmp_trajectory(A, T, S, levels, np.ascontiguousarray(p0.numpy()).reshape(-1),
                                    np.concatenate([canon(x) for x in xi]), u)
        assert abs(info.H0 - ref["H0"]) < 1e-8 * max(1, abs(ref["H0"]))
        assert abs(info.dH - ref["dH"]) < 1e-8, (info.dH, ref["dH"])
        assert bool(info.accepted) == ref["accepted"]
        Ug = np.zeros(lat.V * 72)
        capi.pfmp_gauge_get(g.ctx, Ug, capi.PFMP_HOST)
        assert rel_l2(from_canon(Ug, lat, (4, 3, 3)), ref["U"]) < 1e-10
        # force statistics: every integrated term was evaluated, and its force is non-zero
        for t, l in enumerate(levels):
            assert info.nforce[t] > 0 and info.fmax[t] >= info.favg[t] > 0
        assert sum(info.k_apply_term[t] for t in range(len(levels))) <= info.k_apply
    finally:
        capi.pfmp_action_destroy(A)
        g.close()


def test_mixed_solver_action(world):
    """1PF-2MP with the action's CG in mixed precision (FP32 iterations, FP64-accurate
    true residual, 1e-12): heatbath, every term and the Hasenbusch-ratio forces = oracle."""
    from oracle.action import Action, scheme

    lat, U, g, capi = world
    act = Action(lat, BETA, CSW, KAPPAS, scheme("1PF-2MP", **SCHEMES["1PF-2MP"][3]), mu=MU, nu=NU, tol=TOL)
    d = _def(capi, scheme="1PF-2MP")
    d.solver = capi.PFMP_SOLVER_CG_MIXED
    A = capi.pfmp_action_create_def(g.ctx, d)
    try:
        xi = _noise(lat, len(act.pf), 90)
        phis = act.heatbath(U, xi)
        capi.pfmp_action_heatbath(A, np.concatenate([canon(x) for x in xi]))
        S = capi.pfmp_action_eval(A)
        for i in range(len(act.terms)):
            phi = phis[act.pf.index(i)] if i in act.pf else None
            ref = act.S(U, i, phi).item()
            assert abs(S[i] - ref) < 1e-9 * max(1.0, abs(ref)), (i, S[i], ref)
        for i in (4, 5):   # J_1 J_2^{-1} and J_2 K^{-1}
            F = np.zeros(lat.V * 32)
            capi.pfmp_action_force(A, i, F)
            ref = act.F(U, i, phis[act.pf.index(i)])
            assert rel_l2(torch.tensor(F).reshape(*lat.shape, 4, 8), ref) < 1e-9
    finally:
        capi.pfmp_action_destroy(A)


@pytest.mark.slow
def test_force_balanced_schedule(world):
    """Sec. 2.4: forces measured in one PF-MP trajectory set the step counts of the next
    (F_l h_l = const on the maximal forces), and the cost of three trajectories comes out
    finite (Sec. 3.1)."""
    from oracle.integrator import LAMBDA_2MN
    from oracle.tuning import balance_steps

    lat, U0, g, capi = world
    Ug = np.zeros(lat.V * 72)
    capi.pfmp_gauge_get(g.ctx, Ug, capi.PFMP_HOST)
    A = capi.pfmp_action_create_def(g.ctx, _def(capi, scheme="PF-MP"))
    try:
        levels = [1, 1, 1, 0, 0]
        xi = np.concatenate([canon(x) for x in _noise(lat, 3, 120)])
        mom = np.ascontiguousarray(pin.momenta(DIMS, 121)).reshape(-1)
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(n, 0.5, LAMBDA_2MN) for n in (4, 8)])
        info = capi.pfmp_trajectory(A, T, S, levels, mom, xi, 2.0)     # u = 2: rejected, U kept
        fl = [max(info.fmax[t] for t in range(5) if levels[t] == l) for l in (0, 1)]
        n = capi.pfmp_balance_steps(fl, 4)
        assert n == balance_steps(fl, 4) and 4 in n
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(k, 0.5, LAMBDA_2MN) for k in n])
        acc, nmat, dh = [], [], []
        for k in range(3):
            capi.pfmp_gauge_set(g.ctx, Ug, capi.PFMP_HOST)
            capi.pfmp_action_refresh(A)
            mom = np.ascontiguousarray(pin.momenta(DIMS, 130 + k)).reshape(-1)
            xi = np.concatenate([canon(x) for x in _noise(lat, 3, 140 + 3 * k)])
            r = capi.pfmp_trajectory(A, T, S, levels, mom, xi, float(pin.uniform(150 + k)[0]))
            acc.append(r.accepted)
            nmat.append(r.k_apply)
            dh.append(r.dH)
        c = capi.pfmp_cost(acc, nmat, dh)
        assert np.isfinite(c.nmat) and c.nmat > 0 and np.isfinite(c.exp_mdh)
    finally:
        capi.pfmp_gauge_set(g.ctx, Ug, capi.PFMP_HOST)
        capi.pfmp_action_destroy(A)
