"""The reduced-precision MD path against the oracle at 4^4.

* Multi-shift CG with per-shift stopping: FP64 at 1e-10 against the oracle's solutions
  for the 65 shifts of an order-64 correction term; FP32 (the solver of the FP32 forces)
  to its 1e-6 target, each solution's true residual recomputed by the oracle's K.
* FP32 fermion forces (force_prec = PFMP_F32, solves at md_tol = 1e-6) against the
  oracle's FP64 forces.  Bars from the arithmetic: FP32 products carry ~1e-6 relative
  rounding (amplified ~1e2 by a 12-factor filter chain: 1e-4); a solve stopped at 1e-6
  leaves a solution error up to cond(K) x 1e-6 with cond(K) ~ 20 at kappa 0.12 here
  (bar 5e-4); the gauge and clover-determinant forces are products of a few FP32 links
  (bar 1e-5).  The force of Q = P_64 / P_12 is the small remainder (4e-4 of the P_12
  force here) of 52 chain terms each ~1e4 times larger, so the FP32 rounding (6e-8) is
  amplified by that ratio (measured 2.5e-3 relative, 1e-6 of the P_12 force): bar 1e-2.
* The config-1 trajectory (order-8 PF-MP, two-level 2MN 8 x 2, tau 0.5) with the mixed
  CG in the action and FP64 forces: Delta H within 1e-8 of the oracle's.  With FP32
  forces the MD is a different (still reversible, area-preserving) map: Delta H within
  1e-3 of the oracle's, and forward / flip / forward returns the field to 1e-6 (FP32
  roundings of the force can flip between the two passes, whose fields differ in the
  last bits).
"""
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


def _def(capi, terms, kappas=KAPPAS, solver=0, force_prec=0, md_tol=0.0, tol=TOL):
    d = capi.ActionDef()
    d.beta, d.csw, d.nkappa = BETA, CSW, len(kappas)
    for i, k in enumerate(kappas):
        d.kappa[i] = k
    d.mu, d.nu, d.tol, d.max_iter = MU, NU, tol, 5000
    d.solver, d.force_prec, d.md_tol = solver, force_prec, md_tol
    d.nterms = len(terms)
    for i, t in enumerate(terms):
        d.term[i] = capi.Term(KIND[t.kind], t.a, t.b, t.p1, t.p2)
    return d


def test_multishift_fp64_many_shifts(world):
    from oracle import cheby
    from oracle.dirac import WilsonClover
    from oracle.solvers import multishift_cg

    lat, U, g, capi = world
    W = WilsonClover(lat, U, 0.100, CSW)
    op = g.op(0.100, CSW)
    shifts, _ = cheby.residues(64, MU, NU)          # 65 shifts: -z_k and 0
    b = lat.even * torch.tensor(pin.spinor(DIMS, 78)).reshape(*lat.shape, 4, 3)
    bb = g.pack(b, 0, 0)
    xs = [g.buf(0) for _ in range(len(shifts))]
    info = capi.pfmp_solve_multishift(op, (-shifts).numpy(), xs, bb, 1e-12, 3000)
    assert info.true_rel_res < 1e-11
    ref, _ = multishift_cg(W.K, b, -shifts, tol=1e-13)
    for k in range(len(shifts)):
        assert rel_l2(lat.even * g.unpack(xs[k], 0, 0), ref[k]) < 1e-10, k


@pytest.mark.parametrize("n", [8, 64])
def test_multishift_fp32(world, n):
    from oracle import cheby
    from oracle.dirac import WilsonClover

    lat, U, g, capi = world
    W = WilsonClover(lat, U, 0.100, CSW)
    op = g.op(0.100, CSW)
    shifts, _ = cheby.residues(n, MU, NU)
    sig = (-shifts).numpy()
    b = lat.even * torch.tensor(pin.spinor(DIMS, 79)).reshape(*lat.shape, 4, 3)
    b32 = g.pack(b, 1, 0)
    xs = [g.buf(1) for _ in range(len(sig))]
    info = capi.pfmp_solve_multishift_prec(op, capi.PFMP_F32, sig, xs, b32, 1e-6, 3000)
    assert info.iters > 0
    nb = float(torch.linalg.vector_norm(b))
    for k in range(len(sig)):
        x = lat.even * g.unpack(xs[k], 1, 0)
        r = b - (W.K(x) + complex(sig[k]) * x)
        assert float(torch.linalg.vector_norm(r)) / nb < 5e-6, k


@pytest.mark.parametrize("kind,a,b,p1,p2,tol", [("filter", 1, 0, 0, 12, 1e-4), ("filter", 1, 0, 12, 64, 1e-2),
                                               ("filtercorr", 1, 0, 0, 8, 5e-4), ("ratio", 1, 0, 0, 0, 5e-4),
                                               ("inv", 1, 0, 0, 0, 5e-4), ("gauge", 0, 0, 0, 0, 1e-5),
                                               ("det", 0, 0, 0, 0, 1e-5)],
                         ids=["P12", "Q=P64/P12", "corr8", "ratio", "inv", "gauge", "det"])
def test_fp32_forces(world, kind, a, b, p1, p2, tol):
    from oracle.action import Action, Term

    lat, U, g, capi = world
    t = Term(kind, a=a, b=b, p1=p1, p2=p2)
    act = Action(lat, BETA, CSW, KAPPAS, [t], mu=MU, nu=NU, tol=TOL)
    A = capi.pfmp_action_create_def(g.ctx, _def(capi, [t], solver=1, force_prec=capi.PFMP_F32, md_tol=1e-6))
    try:
        phi = lat.even * torch.tensor(pin.spinor(DIMS, 61)).reshape(*lat.shape, 4, 3)
        if act.pf:
            capi.pfmp_action_set_phi(A, 0, canon(phi))
        F = np.zeros(lat.V * 32)
        capi.pfmp_action_force(A, 0, F)
        ref = act.F(U, 0, phi if act.pf else None)
        err = rel_l2(torch.tensor(F).reshape(*lat.shape, 4, 8), ref)
        assert err < tol, err
    finally:
        capi.pfmp_action_destroy(A)


def test_filter_force_after_larger_filter(world):
    """An order-12 filter force after order-64 ones on the same context, FP32 and FP64: the
    new action's buffers may be recycled device memory holding anything (NaN patterns
    included), and every field the force reads must be written first (a zero coefficient
    never multiplies stale contents)."""
    from oracle.action import Action, Term

    lat, U, g, capi = world
    phi = lat.even * torch.tensor(pin.spinor(DIMS, 61)).reshape(*lat.shape, 4, 3)
    ref = None
    for p1, p2, fp in ((0, 64, capi.PFMP_F32), (0, 64, 0), (0, 12, capi.PFMP_F32), (0, 12, 0)):
        t = Term("filter", a=1, b=0, p1=p1, p2=p2)
        A = capi.pfmp_action_create_def(g.ctx, _def(capi, [t], solver=1, force_prec=fp, md_tol=1e-6))
        try:
            capi.pfmp_action_set_phi(A, 0, canon(phi))
            F = np.zeros(lat.V * 32)
            capi.pfmp_action_force(A, 0, F)
        finally:
            capi.pfmp_action_destroy(A)
        assert np.isfinite(F).all(), (p2, fp)
        if p2 == 12:
            if ref is None:
                ref = Action(lat, BETA, CSW, KAPPAS, [t], mu=MU, nu=NU, tol=TOL).F(U, 0, phi)
            err = rel_l2(torch.tensor(F).reshape(*lat.shape, 4, 8), ref)
            assert err < (1e-4 if fp else 1e-9), (fp, err)


@pytest.fixture(scope="module")
def config1_reference():
    from oracle.action import PFMP, PFMPParams
    from oracle.integrator import merge, trajectory, two_mn

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    prm = dict(beta=5.5, kappa=0.120, kappa_h=0.110, csw=1.0, n=8, mu=1.2, nu=0.9, tol=1e-12)
    act = PFMP(lat, PFMPParams(**prm))
    xi = [torch.tensor(pin.spinor(DIMS, 10 + i)).reshape(*lat.shape, 4, 3) * lat.even for i in range(3)]
    p0 = torch.tensor(pin.momenta(DIMS, 5)).reshape(*lat.shape, 4, 8)
    u = float(pin.uniform(6)[0])
    sched = merge([two_mn(8, 0.5), two_mn(16, 0.5)])
    ref = trajectory(act, U, p0, xi, u, [["polycorr", "hasen"], ["gauge", "det", "poly"]], sched)
    return lat, U, xi, p0, u, ref


def _config1_action(capi, g, solver, force_prec, md_tol):
    d = capi.ActionDef()
    d.beta, d.csw, d.nkappa = 5.5, 1.0, 2
    d.kappa[0], d.kappa[1] = 0.120, 0.110
    d.mu, d.nu, d.tol, d.max_iter = 1.2, 0.9, 1e-12, 5000
    d.solver, d.force_prec, d.md_tol = solver, force_prec, md_tol
    capi.pfmp_action_scheme(capi.PFMP_SCHEME_PFMP, 0, 8, d)
    return capi.pfmp_action_create_def(g.ctx, d)


@pytest.mark.parametrize("force_prec,md_tol,bar", [(0, 0.0, 1e-8), (1, 1e-6, 1e-3)], ids=["f64-forces", "f32-forces"])
def test_config1_trajectory_mixed(config1_reference, force_prec, md_tol, bar):
    from oracle.integrator import LAMBDA_2MN
    from paper_1609_02652_gb300 import capi

    lat, U, xi, p0, u, ref = config1_reference
    g = Gpu(lat, U)
    A = _config1_action(capi, g, capi.PFMP_SOLVER_CG_MIXED, force_prec, md_tol)
    try:
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(8, 0.5, LAMBDA_2MN),
                                         capi.pfmp_schedule_2mn(16, 0.5, LAMBDA_2MN)])
        info = capi.pfmp_trajectory(A, T, S, [1, 1, 1, 0, 0], np.ascontiguousarray(p0.numpy()).reshape(-1),
                                    np.concatenate([canon(x) for x in xi]), u)
        assert abs(info.H0 - ref["H0"]) < 1e-8 * max(1, abs(ref["H0"]))
        assert abs(info.dH - ref["dH"]) < bar, (info.dH, ref["dH"])
    finally:
        capi.pfmp_action_destroy(A)
        g.close()


def test_fp32_force_md_reversibility():
    from oracle.integrator import LAMBDA_2MN
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    A = _config1_action(capi, g, capi.PFMP_SOLVER_CG_MIXED, capi.PFMP_F32, 1e-6)
    try:
        xi = [torch.tensor(pin.spinor(DIMS, 10 + i)).reshape(*lat.shape, 4, 3) * lat.even for i in range(3)]
        capi.pfmp_action_heatbath(A, np.concatenate([canon(x) for x in xi]))
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(n, 0.2, LAMBDA_2MN) for n in (2, 4)])
        levels = [1, 1, 1, 0, 0]
        U0 = np.zeros(lat.V * 72)
        capi.pfmp_gauge_get(g.ctx, U0, capi.PFMP_HOST)
        p0 = np.ascontiguousarray(pin.momenta(DIMS, 5)).reshape(-1).copy()
        p = p0.copy()
        capi.pfmp_md(A, T, S, levels, p)
        p = -p
        capi.pfmp_md(A, T, S, levels, p)
        U2 = np.zeros(lat.V * 72)
        capi.pfmp_gauge_get(g.ctx, U2, capi.PFMP_HOST)
        assert np.abs(U2 - U0).max() < 1e-6
        assert np.abs(p + p0).max() < 1e-5
    finally:
        capi.pfmp_action_destroy(A)
        g.close()
