"""GPU solves against the oracle: FP64 CG, mixed FP32/FP64-reliable-update CG and the
same with the stencil on FP16 storage reach a true relative residual below 1e-10,
recomputed by the ORACLE's K on the GPU's solution, and agree with the oracle's own CG
solution."""
import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, canon, from_canon, oracle_gauge, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,eps,kappa", [((4, 4, 4, 8), 0.3, 0.125), ((6, 4, 4, 6), 0.5, 0.130)])
@pytest.mark.parametrize("method", [0, 1, 2], ids=["cg64", "mixed", "half"])
def test_solve_true_residual(dims, eps, kappa, method):
    from oracle.dirac import WilsonClover
    from oracle.solvers import cg
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(dims, eps, 21)
    g = Gpu(lat, U)
    try:
        op = g.op(kappa, 1.0)
        b = lat.even * torch.tensor(pin.spinor(dims, 100)).reshape(*lat.shape, 4, 3)
        bb = g.pack(b, 0, 0)
        xx = g.buf(0)
        prm = capi.SolverParams(method=method, tol=1e-10, max_iter=5000, delta=0.1, check_every=8)
        info = capi.pfmp_solve(op, prm, xx, bb)
        x = lat.even * g.unpack(xx, 0, 0)
        W = WilsonClover(lat, U, kappa, 1.0)
        r = b - W.K(x)
        true_res = float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b))
        assert true_res < 1e-10
        assert abs(true_res - info.true_rel_res) < 1e-11
        xo, _, _ = cg(W.K, b, tol=1e-12)
        assert rel_l2(x, xo) < 1e-8
        if method >= 1:
            assert info.reliable_updates >= 1
    finally:
        g.close()


def test_solve_host_path_and_errors():
    from oracle.dirac import WilsonClover
    from paper_1609_02652_gb300 import capi

    dims = (4, 4, 4, 4)
    lat, U = oracle_gauge(dims, 0.3, 1)
    g = Gpu(lat, U)
    try:
        op = g.op(0.12, 1.0)
        b = lat.even * torch.tensor(pin.spinor(dims, 3)).reshape(*lat.shape, 4, 3)
        x = np.zeros(lat.V * 24)
        prm = capi.SolverParams(method=1, tol=1e-10, max_iter=1000, delta=0.1, check_every=8)
        info = capi.pfmp_solve_host(op, prm, x, canon(b))
        xs = from_canon(x, lat, (4, 3))
        W = WilsonClover(lat, U, 0.12, 1.0)
        res = float(torch.linalg.vector_norm(b - W.K(xs)) / torch.linalg.vector_norm(b))
        assert res < 1e-10 and info.status == 0
        assert (lat.odd * xs).abs().max() == 0
        # iteration cap -> PFMP_E_NOT_CONVERGED with a usable residual report
        prm = capi.SolverParams(method=0, tol=1e-10, max_iter=2, delta=0.1, check_every=1)
        info = capi.pfmp_solve_host(op, prm, x, canon(b), raise_on_error=False)
        assert info.status == capi.PFMP_E_NOT_CONVERGED and info.true_rel_res > 1e-10
        # zero right-hand side -> x = 0 at once
        info = capi.pfmp_solve_host(op, prm, x, np.zeros(lat.V * 24))
        assert info.status == 0 and np.abs(x).max() == 0
        # invalid arguments are rejected with a status, not a crash
        with pytest.raises(capi.PfmpError):
            capi.pfmp_ctx_create((4, 4, 3, 4), -1)
    finally:
        g.close()


def test_fp64_cg_full_size_matches_oracle_iterations():
    """At the benchmark size (16^3 x 32) the FP64 CG on the GPU takes the oracle's number of
    iterations (stored by tests/golden/make_cg_iterations.py) to reach 1e-10, +-2 for the
    different summation order, and its true residual agrees with the oracle's."""
    import json
    import os

    from paper_1609_02652_gb300 import capi

    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cg_iterations_16x16x16x32.json")))
    dims = tuple(gold["dims"])
    ctx = capi.pfmp_ctx_create(dims, -1, None)
    try:
        h = np.ascontiguousarray(pin.gauge_algebra(dims, 1)).reshape(-1)
        capi.pfmp_gauge_from_algebra(ctx, h, gold["eps"], capi.PFMP_HOST)
        op = capi.pfmp_op_create(ctx, gold["kappa"], gold["csw"])
        b = np.ascontiguousarray(pin.spinor(dims, 100)).view(np.float64).reshape(-1)
        x = np.zeros_like(b)
        for method in (0, 1):
            prm = capi.SolverParams(method=method, tol=gold["tol"], max_iter=2000, delta=0.1, check_every=8)
            info = capi.pfmp_solve_host(op, prm, x, b)
            assert info.true_rel_res < 1e-10
            if method == 0:
                assert abs(info.iters - gold["iterations"]) <= 2
                assert abs(info.true_rel_res - gold["true_rel_res"]) < 0.05 * gold["true_rel_res"]
        capi.pfmp_op_destroy(op)
    finally:
        capi.pfmp_ctx_destroy(ctx)


def test_double_float_true_residual():
    """The double-float residual b - K x (FP32-pair arithmetic) agrees with the FP64 one and
    with the oracle's, both for an O(1) residual and for a converged solution."""
    from oracle.dirac import WilsonClover
    from paper_1609_02652_gb300 import capi

    dims = (6, 4, 4, 8)
    lat, U = oracle_gauge(dims, 0.5, 7)
    g = Gpu(lat, U)
    try:
        op = g.op(0.13, 1.0)
        W = WilsonClover(lat, U, 0.13, 1.0)
        b = lat.even * torch.tensor(pin.spinor(dims, 5)).reshape(*lat.shape, 4, 3)
        x = lat.even * torch.tensor(pin.spinor(dims, 6)).reshape(*lat.shape, 4, 3)
        bb, xx = g.pack(b, 0, 0), g.pack(x, 0, 0)
        r64, rdf = g.buf(0), g.buf(0)
        capi.pfmp_true_residual(op, capi.PFMP_F64, r64, xx, bb)
        capi.pfmp_true_residual(op, capi.PFMP_DF, rdf, xx, bb)
        ref = b - W.K(x)
        scale = float(torch.linalg.vector_norm(W.K(x)))
        assert float(torch.linalg.vector_norm(lat.even * g.unpack(rdf, 0, 0) - ref)) < 1e-12 * scale
        assert float(torch.linalg.vector_norm(lat.even * g.unpack(r64, 0, 0) - ref)) < 1e-13 * scale
        # converged x: the residual itself is ~1e-11 |b| and must still be resolved
        prm = capi.SolverParams(method=0, tol=1e-11, max_iter=4000, delta=0.1, check_every=8)
        capi.pfmp_solve(op, prm, xx, bb)
        xs = lat.even * g.unpack(xx, 0, 0)
        ref = b - W.K(xs)
        rel_df = capi.pfmp_true_residual(op, capi.PFMP_DF, rdf, xx, bb)
        rel_ref = float(torch.linalg.vector_norm(ref) / torch.linalg.vector_norm(b))
        assert abs(rel_df - rel_ref) < 0.05 * rel_ref + 1e-13
        assert float(torch.linalg.vector_norm(lat.even * g.unpack(rdf, 0, 0) - ref)) < 1e-13 * float(torch.linalg.vector_norm(b))
    finally:
        g.close()
