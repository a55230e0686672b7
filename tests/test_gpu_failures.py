"""Failure paths of the C-ABI, made on the host (no fault is provoked on the GPU): a NaN
in a right-hand side, in a gauge field or in the momenta returns PFMP_E_NAN from the
solver, the operator build, the multi-shift solver and the trajectory, and a failed
trajectory leaves the gauge field as it was; shifts that can make K + sigma singular are
refused; FGCR with a preconditioner that cannot reduce the residual falls back to the
mixed CG and still reaches 1e-10 (judged by the oracle's K)."""
import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, canon, from_canon, oracle_gauge

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 8)


def test_nan_right_hand_side():
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    try:
        op = g.op(0.12, 1.0)
        b = lat.even * torch.tensor(pin.spinor(DIMS, 3)).reshape(*lat.shape, 4, 3)
        bb = g.pack(b, 0, 0)
        bb[17] = float("nan")
        x = g.buf(0)
        for method in (0, 1, 2):
            prm = capi.SolverParams(method=method, tol=1e-10, max_iter=500, delta=0.1, check_every=8)
            st = capi.lib().pfmp_solve(op, capi.C.byref(prm), capi._ptr(x), capi._ptr(bb), None)
            assert st == capi.PFMP_E_NAN, (method, st)
        with pytest.raises(capi.PfmpError) as e:
            capi.pfmp_solve_multishift(op, [0.1 + 0.2j, 0.0], [g.buf(0), g.buf(0)], bb, 1e-10, 500)
        assert e.value.status == capi.PFMP_E_NAN
    finally:
        g.close()


def test_nan_gauge_field():
    """A NaN link reaches the clover field strength of its four plaquettes, so building
    the operator fails in the Cholesky factorisation of A = 1 - kappa c_sw sum sigma F,
    with a clover term and without one (0 x NaN is NaN)."""
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    Ubad = U.clone()
    Ubad[1, 2, 3, 1, 2, 0, 1] = complex(float("nan"), 0.0)
    g = Gpu(lat, Ubad)
    try:
        for csw in (1.0, 0.0):
            with pytest.raises(capi.PfmpError) as e:
                g.op(0.12, csw)
            assert e.value.status == capi.PFMP_E_NAN, csw
    finally:
        g.close()


def test_nan_momenta_in_trajectory():
    from oracle.integrator import LAMBDA_2MN
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    ap = capi.ActionParams(beta=5.5, kappa=0.12, kappa_h=0.11, csw=1.0, n=4, mu=1.2, nu=0.9, tol=1e-10,
                           max_iter=2000)
    A = capi.pfmp_action_create(g.ctx, ap)
    try:
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(2, 0.1, LAMBDA_2MN)])
        xi = np.concatenate([canon(lat.even * torch.tensor(pin.spinor(DIMS, 10 + i)).reshape(*lat.shape, 4, 3))
                             for i in range(3)])
        mom = np.ascontiguousarray(pin.momenta(DIMS, 5)).reshape(-1).copy()
        mom[100] = np.nan
        with pytest.raises(capi.PfmpError) as e:
            capi.pfmp_trajectory(A, T, S, [0, 0, 0, 0, 0], mom, xi, 0.5)
        assert e.value.status == capi.PFMP_E_NAN
        # the failed trajectory left the gauge field as it was, and the action is usable
        Ug = np.zeros(lat.V * 72)
        capi.pfmp_gauge_get(g.ctx, Ug, capi.PFMP_HOST)
        assert np.array_equal(Ug, canon(U))
        mom[100] = 0.0
        info = capi.pfmp_trajectory(A, T, S, [0, 0, 0, 0, 0], mom, xi, 0.5)
        assert np.isfinite(info.dH)
    finally:
        capi.pfmp_action_destroy(A)
        g.close()


@pytest.mark.parametrize("sigma", [-0.05 + 0.0j, complex(float("nan"), 0.0), complex(0.1, float("inf"))],
                         ids=["negative-real", "nan", "inf"])
def test_singular_or_invalid_shift_refused(sigma):
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    try:
        op = g.op(0.12, 1.0)
        b = g.pack(lat.even * torch.tensor(pin.spinor(DIMS, 3)).reshape(*lat.shape, 4, 3), 0, 0)
        with pytest.raises(capi.PfmpError) as e:
            capi.pfmp_solve_multishift(op, [0.2 - 0.1j, sigma], [g.buf(0), g.buf(0)], b, 1e-10, 500)
        assert e.value.status == capi.PFMP_E_INVALID
        # complex and non-negative real shifts are accepted
        info = capi.pfmp_solve_multishift(op, [0.2 - 0.1j, 0.0, 0.3], [g.buf(0) for _ in range(3)], b, 1e-10, 500)
        assert info.true_rel_res < 1e-9
    finally:
        g.close()


def test_fgcr_falls_back_to_cg():
    """A one-layer network whose only weight is the chiral projector (1 + g5)/2 on the site
    term: K N has half rank, FGCR stalls near 1/sqrt(2) of |b|, and after two outer passes
    without a 10% gain the mixed CG finishes the solve."""
    from oracle.dirac import WilsonClover
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    nn = capi.pfmp_nn_create(g.ctx, [1, 1])
    try:
        op = g.op(0.125, 1.0)
        w = np.zeros((9, 1, 1, 4, 4), dtype=np.complex128)
        w[0, 0, 0] = np.diag([1.0, 1.0, 0.0, 0.0])
        capi.pfmp_nn_set_weights(nn, [w])
        b = lat.even * torch.tensor(pin.spinor(DIMS, 8)).reshape(*lat.shape, 4, 3)
        bb, x = g.pack(b, 0, 0), g.buf(0)
        prm = capi.SolverParams(method=1, tol=1e-10, max_iter=4000, delta=0.1, check_every=8, restart=8)
        info = capi.pfmp_solve_fgcr(op, nn, prm, x, bb)
        assert info.status == 0 and info.reliable_updates > 0      # fallback CG iterations
        xs = lat.even * g.unpack(x, 0, 0)
        W = WilsonClover(lat, U, 0.125, 1.0)
        res = float(torch.linalg.vector_norm(b - W.K(xs)) / torch.linalg.vector_norm(b))
        assert res < 1e-10 and abs(res - info.true_rel_res) < 1e-11
    finally:
        capi.pfmp_nn_destroy(nn)
        g.close()


def test_fma_rate_probe_and_trajectory_timings():
    """pfmp_fma_rate measures the FP64 and FP32 FMA pipes (an FP32 rate many times the
    FP64 rate on this part); a trajectory reports positive wall times per term's forces and
    for the link updates, which add up to no more than the whole call."""
    from oracle.integrator import LAMBDA_2MN
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(DIMS, 0.3, 1)
    g = Gpu(lat, U)
    try:
        r64 = capi.pfmp_fma_rate(g.ctx, capi.PFMP_F64)
        r32 = capi.pfmp_fma_rate(g.ctx, capi.PFMP_F32)
        assert 0.05 < r64 < 1e3 and 1.0 < r32 < 1e4 and r32 > 8 * r64, (r64, r32)
        with pytest.raises(capi.PfmpError):
            capi.pfmp_fma_rate(g.ctx, capi.PFMP_H16)
        ap = capi.ActionParams(beta=5.5, kappa=0.12, kappa_h=0.11, csw=1.0, n=4, mu=1.2, nu=0.9, tol=1e-10,
                               max_iter=2000)
        A = capi.pfmp_action_create(g.ctx, ap)
        try:
            T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(2, 0.1, LAMBDA_2MN)])
            xi = np.concatenate([canon(lat.even * torch.tensor(pin.spinor(DIMS, 10 + i)).reshape(*lat.shape, 4, 3))
                                 for i in range(3)])
            mom = np.ascontiguousarray(pin.momenta(DIMS, 5)).reshape(-1)
            info = capi.pfmp_trajectory(A, T, S, [0, 0, 0, 0, 0], mom, xi, 0.5)
            per_term = [info.ms_force[t] for t in range(5)]
            assert all(v > 0 for v in per_term) and info.ms_update > 0
            assert sum(per_term) + info.ms_update <= info.ms_total
        finally:
            capi.pfmp_action_destroy(A)
    finally:
        g.close()
