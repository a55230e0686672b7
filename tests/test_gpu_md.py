"""GPU parity of the PF-MP machinery against the oracle at 4^4 (FP64): multi-shift CG
with complex shifts, the polynomial filter and its half product, the heatbath, each
action term, each force term, and one full trajectory (config: eps = 0.3, c_sw = 1.0,
kappa = 0.120, kappa' = 0.110, order-8 filter, 2-level Omelyan 8 x 2 steps, tau = 0.5,
CG to 1e-12): Delta H within 1e-8 of the oracle's."""
import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, canon, from_canon, oracle_gauge, rel_l2

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
PRM = dict(beta=5.5, kappa=0.120, kappa_h=0.110, csw=1.0, n=8, mu=1.2, nu=0.9, tol=1e-12)


def _action(capi, g, **over):
    p = dict(PRM, **over)
    ap = capi.ActionParams(beta=p["beta"], kappa=p["kappa"], kappa_h=p["kappa_h"], csw=p["csw"], n=p["n"],
                           mu=p["mu"], nu=p["nu"], tol=p["tol"], max_iter=5000)
    return capi.pfmp_action_create(g.ctx, ap)


@pytest.fixture(scope="module")
def world():
    from oracle.action import PFMP, PFMPParams
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    act = PFMP(lat, PFMPParams(**PRM))
    xi = [torch.tensor(pin.spinor(DIMS, 10 + i)).reshape(*lat.shape, 4, 3) * lat.even for i in range(3)]
    phis = act.heatbath(U, *xi)
    A = _action(capi, g)
    yield lat, U, g, capi, act, xi, phis, A
    capi.pfmp_action_destroy(A)
    g.close()


def test_multishift_complex_shifts(world):
    from oracle import cheby
    from oracle.dirac import WilsonClover
    from oracle.solvers import multishift_cg

    lat, U, g, capi, *_ = world
    W = WilsonClover(lat, U, 0.110, 1.0)
    op = g.op(0.110, 1.0)
    shifts, _ = cheby.residues(8, 1.2, 0.9)
    b = lat.even * torch.tensor(pin.spinor(DIMS, 77)).reshape(*lat.shape, 4, 3)
    bb = g.pack(b, 0, 0)
    xs = [g.buf(0) for _ in range(len(shifts))]
    info = capi.pfmp_solve_multishift(op, (-shifts).numpy(), xs, bb, 1e-12, 2000)
    assert info.true_rel_res < 1e-11
    ref, _ = multishift_cg(W.K, b, -shifts, tol=1e-13)
    for k in range(len(shifts)):
        got = lat.even * g.unpack(xs[k], 0, 0)
        assert rel_l2(got, ref[k]) < 1e-10


def test_poly_and_half_product(world):
    from oracle import cheby
    from oracle.dirac import WilsonClover

    lat, U, g, capi, *_ = world
    W = WilsonClover(lat, U, 0.110, 1.0)
    op = g.op(0.110, 1.0)
    z, an = capi.pfmp_poly_roots(8, 1.2, 0.9)
    assert np.allclose(z, cheby.roots(8, 1.2, 0.9).numpy(), atol=1e-15)
    assert abs(an - cheby.norm(8, 1.2, 0.9)) < 1e-15 * an
    v = lat.even * torch.tensor(pin.spinor(DIMS, 5)).reshape(*lat.shape, 4, 3)
    bi, bo = g.pack(v, 0, 0), g.buf(0)
    for which, ref in [(0, cheby.apply_poly(W.K, v, 8, 1.2, 0.9)), (1, cheby.apply_R(W.K, v, 8, 1.2, 0.9)),
                       (2, cheby.apply_R(W.K, v, 8, 1.2, 0.9, dagger=True))]:
        capi.pfmp_poly_apply(op, 8, 1.2, 0.9, which, bo, bi)
        assert rel_l2(lat.even * g.unpack(bo, 0, 0), ref) < 1e-13
    with pytest.raises(capi.PfmpError):
        capi.pfmp_poly_apply(op, 7, 1.2, 0.9, 0, bo, bi)


def test_heatbath_and_action(world):
    lat, U, g, capi, act, xi, phis, A = world
    capi.pfmp_action_heatbath(A, np.concatenate([canon(x) for x in xi]))
    for i in range(3):
        out = np.zeros(lat.V * 24)
        capi.pfmp_action_get_phi(A, i, out)
        assert rel_l2(lat.even * from_canon(out, lat, (4, 3)), phis[i]) < 1e-10
    S = capi.pfmp_action_eval(A)
    ref = [act.S_gauge(U).item(), act.S_det(U).item(), act.S_poly(U, phis[0]).item(),
           act.S_polycorr(U, phis[1]).item(), act.S_hasen(U, phis[2]).item()]
    for t in range(5):
        assert abs(S[t] - ref[t]) < 1e-9 * max(1.0, abs(ref[t])), (t, S[t], ref[t])
    for i in range(3):   # heatbath identity S_i(phi_i) = xi_i^dag xi_i
        assert abs(S[2 + i] - (xi[i].abs() ** 2).sum().item()) < 1e-9 * S[2 + i]


@pytest.mark.parametrize("term,tol", [(0, 1e-12), (1, 1e-11), (2, 1e-11), (3, 1e-9), (4, 1e-9)],
                         ids=["gauge", "det", "poly", "polycorr", "hasen"])
def test_force_terms(world, term, tol):
    lat, U, g, capi, act, xi, phis, A = world
    for i in range(3):
        capi.pfmp_action_set_phi(A, i, canon(phis[i]))
    F = np.zeros(lat.V * 32)
    capi.pfmp_action_force(A, term, F)
    got = torch.tensor(F).reshape(*lat.shape, 4, 8)
    ref = [act.F_gauge(U), act.F_det(U), act.F_poly(U, phis[0]), act.F_polycorr(U, phis[1]),
           act.F_hasen(U, phis[2])][term]
    assert rel_l2(got, ref) < tol


@pytest.mark.slow
def test_trajectory_delta_h_matches_oracle():
    from oracle.action import PFMP, PFMPParams
    from oracle.integrator import LAMBDA_2MN, merge, trajectory, two_mn
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    act = PFMP(lat, PFMPParams(**PRM))
    xi = [torch.tensor(pin.spinor(DIMS, 10 + i)).reshape(*lat.shape, 4, 3) * lat.even for i in range(3)]
    p0 = torch.tensor(pin.momenta(DIMS, 5)).reshape(*lat.shape, 4, 8)
    u = float(pin.uniform(6)[0])
    tau = 0.5
    sched = merge([two_mn(8, tau), two_mn(16, tau)])
    levels = [["polycorr", "hasen"], ["gauge", "det", "poly"]]
    ref = trajectory(act, U, p0, xi, u, levels, sched)

    g = Gpu(lat, U)
    A = _action(capi, g)
    try:
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(8, tau, LAMBDA_2MN),
                                         capi.pfmp_schedule_2mn(16, tau, LAMBDA_2MN)])
        # term -> level: gauge, det, poly on the fine level (1); polycorr, hasen coarse (0)
        info = capi.pfmp_trajectory(A, T, S, [1, 1, 1, 0, 0], np.ascontiguousarray(p0.numpy()).reshape(-1),
                                    np.concatenate([canon(x) for x in xi]), u)
        assert abs(info.H0 - ref["H0"]) < 1e-8 * max(1, abs(ref["H0"]))
        assert abs(info.dH - ref["dH"]) < 1e-8, (info.dH, ref["dH"])
        assert bool(info.accepted) == ref["accepted"]
        Ug = np.zeros(lat.V * 72)
        capi.pfmp_gauge_get(g.ctx, Ug, capi.PFMP_HOST)
        Uref = ref["U"]
        assert rel_l2(from_canon(Ug, lat, (4, 3, 3)), Uref) < 1e-10
    finally:
        capi.pfmp_action_destroy(A)
        g.close()


def test_md_reversibility():
    """App. B: the merged 2MN scheme is time reversible -- MD forward, momenta flipped, MD
    forward again returns the gauge field and the negated momenta (FP64, CG to 1e-12)."""
    from oracle.integrator import LAMBDA_2MN
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    A = _action(capi, g)
    try:
        xi = [torch.tensor(pin.spinor(DIMS, 10 + i)).reshape(*lat.shape, 4, 3) * lat.even for i in range(3)]
        capi.pfmp_action_heatbath(A, np.concatenate([canon(x) for x in xi]))
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(n, 0.1, LAMBDA_2MN) for n in (2, 3)])
        levels = [1, 1, 1, 0, 0]
        U0 = np.zeros(lat.V * 72)
        capi.pfmp_gauge_get(g.ctx, U0, capi.PFMP_HOST)
        p0 = np.ascontiguousarray(pin.momenta(DIMS, 5)).reshape(-1).copy()
        p = p0.copy()
        capi.pfmp_md(A, T, S, levels, p)
        U1 = np.zeros(lat.V * 72)
        capi.pfmp_gauge_get(g.ctx, U1, capi.PFMP_HOST)
        assert np.abs(U1 - U0).max() > 1e-3          # the field did move
        p = -p
        capi.pfmp_md(A, T, S, levels, p)
        U2 = np.zeros(lat.V * 72)
        capi.pfmp_gauge_get(g.ctx, U2, capi.PFMP_HOST)
        assert np.abs(U2 - U0).max() < 1e-11
        assert np.abs(p + p0).max() < 1e-10
    finally:
        capi.pfmp_action_destroy(A)
        g.close()


@pytest.mark.slow
def test_exp_minus_delta_h_is_one():
    """<exp(-dH)> = 1 over an HMC chain (area preservation and reversibility of the MD):
    gauge action plus clover determinant at 4^4 (no pseudofermions, so many trajectories
    are cheap), beta 5.5, 2MN 6 steps over tau 0.5; 60 trajectories to thermalise from
    the synthetic start, then 300 measured; the mean within 4 autocorrelation-corrected
    standard errors of 1 (tau_int taken as 10)."""
    from oracle.integrator import LAMBDA_2MN
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    d = capi.ActionDef()
    d.beta, d.csw, d.nkappa = 5.5, 1.0, 1
    d.kappa[0] = 0.120
    d.mu, d.nu, d.tol, d.max_iter = 1.2, 0.9, 1e-12, 5000
    d.nterms = 2
    d.term[0] = capi.Term(capi.PFMP_KIND_GAUGE, 0, 0, 0, 0)
    d.term[1] = capi.Term(capi.PFMP_KIND_DET, 0, 0, 0, 0)
    A = capi.pfmp_action_create_def(g.ctx, d)
    try:
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(6, 0.5, LAMBDA_2MN)])
        dummy = np.zeros(1)
        ex = []
        for k in range(360):
            mom = np.ascontiguousarray(pin.momenta(DIMS, 1000 + k)).reshape(-1)
            uk = float(pin.uniform(2000 + k)[0])
            info = capi.pfmp_trajectory(A, T, S, [0, 0], mom, dummy, uk)
            if k >= 60:
                ex.append(np.exp(-info.dH))
        ex = np.array(ex)
        err = np.sqrt(2 * 10.0) * ex.std(ddof=1) / np.sqrt(len(ex))
        assert abs(ex.mean() - 1.0) < 4 * err + 1e-12, (ex.mean(), err)
    finally:
        capi.pfmp_action_destroy(A)
        g.close()


def test_exp_minus_delta_h_is_one_with_fermion_terms():
    """<exp(-dH)> = 1 over an HMC chain carrying every PF-MP term (gauge, clover
    determinant, filter P_4(J), filter correction [J P_4(J)]^{-1}, Hasenbusch ratio
    J K^{-1}) at 4^4: beta 5.5, kappa 0.120, kappa' 0.110, two-level 2MN (2 steps for the
    correction and ratio terms, 4 for the rest) over tau 0.5, CG to 1e-10; 40 trajectories
    to thermalise from the synthetic start, then 200 measured; the mean within 4
    autocorrelation-corrected standard errors of 1 (tau_int taken as 10)."""
    from oracle.integrator import LAMBDA_2MN
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    A = _action(capi, g, n=4, tol=1e-10)
    try:
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(2, 0.5, LAMBDA_2MN),
                                         capi.pfmp_schedule_2mn(4, 0.5, LAMBDA_2MN)])
        levels = [1, 1, 1, 0, 0]
        ex, acc = [], []
        for k in range(240):
            mom = np.ascontiguousarray(pin.momenta(DIMS, 4000 + k)).reshape(-1)
            xi = np.concatenate([canon(lat.even * torch.tensor(pin.spinor(DIMS, 9000 + 3 * k + i)).reshape(
                *lat.shape, 4, 3)) for i in range(3)])
            info = capi.pfmp_trajectory(A, T, S, levels, mom, xi, float(pin.uniform(7000 + k)[0]))
            if k >= 40:
                ex.append(np.exp(-info.dH))
                acc.append(info.accepted)
        ex = np.array(ex)
        err = np.sqrt(2 * 10.0) * ex.std(ddof=1) / np.sqrt(len(ex))
        assert ex.std() > 1e-3                                  # dH is not trivially zero
        assert abs(ex.mean() - 1.0) < 4 * err + 1e-12, (ex.mean(), err)
        assert np.mean(acc) > 0.5
    finally:
        capi.pfmp_action_destroy(A)
        g.close()
