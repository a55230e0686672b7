"""GPU parity of the large filters against the oracle at 4^4 (FP64): the filter P_n(J)
and its half products at the orders of the production action (12, 48, 64; App. A), the
filter force (App. C eq. force_poly) at orders 12 and 48 and for the factorised
Q = P_64 / P_12, and the correction force (eq. force_polycorr: one multi-shift solve
with n + 1 = 49 and 65 complex shifts).  Both sides apply the root factors in the order
k = 1..n; the bars allow for the rounding that order accumulates at high n (the oracle's
own pin against a dense eigendecomposition measures 2e-13 at n = 48, 4e-12 at 64)."""
import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, canon, from_canon, oracle_gauge, rel_l2

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
KAPPAS = [0.120, 0.100, 0.110]
BETA, CSW, MU, NU, TOL = 5.5, 1.0, 1.2, 0.9, 1e-12
KIND = {"gauge": 0, "det": 1, "filter": 2, "filtercorr": 3, "ratio": 4, "inv": 5}


@pytest.fixture(scope="module")
def world():
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    yield lat, U, g, capi
    g.close()


def _def(capi, terms):
    d = capi.ActionDef()
    d.beta, d.csw, d.nkappa = BETA, CSW, len(KAPPAS)
    for i, k in enumerate(KAPPAS):
        d.kappa[i] = k
    d.mu, d.nu, d.tol, d.max_iter = MU, NU, TOL, 5000
    d.nterms = len(terms)
    for i, t in enumerate(terms):
        d.term[i] = capi.Term(KIND[t.kind], t.a, t.b, t.p1, t.p2)
    return d


@pytest.mark.parametrize("n,bar", [(12, 1e-13), (48, 1e-11), (64, 1e-10)])
def test_poly_high_order(world, n, bar):
    from oracle import cheby
    from oracle.dirac import WilsonClover

    lat, U, g, capi = world
    W = WilsonClover(lat, U, 0.100, CSW)
    op = g.op(0.100, CSW)
    z, an = capi.pfmp_poly_roots(n, MU, NU)
    assert np.allclose(z, cheby.roots(n, MU, NU).numpy(), atol=1e-14)
    assert abs(an - cheby.norm(n, MU, NU)) < 1e-13 * an
    v = lat.even * torch.tensor(pin.spinor(DIMS, 7)).reshape(*lat.shape, 4, 3)
    bi, bo = g.pack(v, 0, 0), g.buf(0)
    for which, ref in [(0, cheby.apply_poly(W.K, v, n, MU, NU)), (1, cheby.apply_R(W.K, v, n, MU, NU)),
                       (2, cheby.apply_R(W.K, v, n, MU, NU, dagger=True))]:
        capi.pfmp_poly_apply(op, n, MU, NU, which, bo, bi)
        assert rel_l2(lat.even * g.unpack(bo, 0, 0), ref) < bar, (n, which)


# Bars.  Filter forces: the oracle forms the chains eta_i, chi_i in index order k = 1..n
# (the paper's), the library in bit-reversed order; each side's rounding is amplified by
# the size of its partial products, which for the 52 factors of Q = P_64 / P_12 in index
# order reach ~1e9 times the final product (a bound; measured: 4e-9 between the two
# sides): bar 5e-8.  Correction forces: at (mu, nu) = (1.2, 0.9) an order-48 filter
# reproduces 1/J to ~1e-17 on this spectrum, [J P(J)]^{-1} is the identity to rounding
# and its force (|F| ~ 1e-11) is rounding noise; on the narrower ellipse nu = 1.19 the
# approximation error is 3e-3 (48) and 2e-4 (64) and the correction force is O(0.1-1),
# sensitive to the solver tolerance (1e-12) at 1e-11: bar 1e-9.
@pytest.mark.parametrize("kind,p1,p2,nu,tol", [("filter", 0, 12, NU, 1e-11), ("filter", 0, 48, NU, 1e-10),
                                              ("filter", 12, 64, NU, 5e-8), ("filtercorr", 0, 48, 1.19, 1e-9),
                                              ("filtercorr", 0, 64, 1.19, 1e-9)],
                         ids=["P12", "P48", "Q=P64/P12", "corr48", "corr64"])
def test_high_order_forces(world, kind, p1, p2, nu, tol):
    from oracle.action import Action, Term

    lat, U, g, capi = world
    t = Term(kind, a=1, p1=p1, p2=p2)
    act = Action(lat, BETA, CSW, KAPPAS, [t], mu=MU, nu=nu, tol=TOL)
    d = _def(capi, [t])
    d.nu = nu
    A = capi.pfmp_action_create_def(g.ctx, d)
    try:
        phi = lat.even * torch.tensor(pin.spinor(DIMS, 61)).reshape(*lat.shape, 4, 3)
        capi.pfmp_action_set_phi(A, 0, canon(phi))
        F = np.zeros(lat.V * 32)
        capi.pfmp_action_force(A, 0, F)
        ref = act.F(U, 0, phi)
        assert rel_l2(torch.tensor(F).reshape(*lat.shape, 4, 8), ref) < tol
    finally:
        capi.pfmp_action_destroy(A)


def test_production_terms_heatbath_and_action(world):
    """The term list of the 24^3 x 48 production run (P_12(J_1), Q = P_64/P_12 (J_1),
    [J_1 P_64(J_1)]^{-1}, J_1 J_2^{-1}, J_2 K^{-1}, with kappa_1 < kappa_2 < kappa) at 4^4:
    every pseudofermion and action value equals the oracle's, and each S_i(phi_i) is
    xi_i^dag xi_i.  The Q filter's heatbath sums partial fractions over its 26 roots with
    Im < 0; those roots lie close together along the ellipse, the residues are large and
    cancel, and each side's multi-shift tolerance (1e-12) is amplified to ~1e-8 (measured
    8.8e-9 between the two): bar 1e-7 for that pseudofermion, 1e-10 for the others."""
    from oracle.action import Action, Term

    lat, U, g, capi = world
    kap = [0.120, 0.100, 0.110]
    terms = [Term("gauge"), Term("det"), Term("filter", a=1, p2=12), Term("filter", a=1, p1=12, p2=64),
             Term("filtercorr", a=1, p2=64), Term("ratio", a=1, b=2), Term("ratio", a=2, b=0)]
    act = Action(lat, BETA, CSW, kap, terms, mu=MU, nu=NU, tol=TOL)
    A = capi.pfmp_action_create_def(g.ctx, _def(capi, terms))
    try:
        nt, npf = capi.pfmp_action_counts(A)
        assert (nt, npf) == (7, 5)
        xi = [lat.even * torch.tensor(pin.spinor(DIMS, 90 + k)).reshape(*lat.shape, 4, 3) for k in range(npf)]
        phis = act.heatbath(U, xi)
        capi.pfmp_action_heatbath(A, np.concatenate([canon(x) for x in xi]))
        bar = [1e-10, 1e-7, 1e-10, 1e-10, 1e-10]   # pseudofermion 1: the Q filter
        for k in range(npf):
            out = np.zeros(lat.V * 24)
            capi.pfmp_action_get_phi(A, k, out)
            assert rel_l2(lat.even * from_canon(out, lat, (4, 3)), phis[k]) < bar[k], k
        S = capi.pfmp_action_eval(A)
        for i in range(nt):
            phi = phis[act.pf.index(i)] if i in act.pf else None
            ref = act.S(U, i, phi).item()
            assert abs(S[i] - ref) < 1e-9 * max(1.0, abs(ref)), (i, S[i], ref)
        for k, i in enumerate(act.pf):
            assert abs(S[i] - (xi[k].abs() ** 2).sum().item()) < 10 * bar[k] * S[i]
    finally:
        capi.pfmp_action_destroy(A)
