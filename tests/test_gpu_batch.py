"""Batched multi-system, multi-RHS mixed-precision solves (one persistent cooperative
launch with bounded grid barriers): every right-hand side reaches a true relative residual
below 1e-10, recomputed by the ORACLE's K on the GPU solution, and matches the
single-system solver; the barrier's bounded wait and a NaN right-hand side give their
status codes."""
import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, oracle_gauge, rel_l2

pytestmark = pytest.mark.gpu

SYSTEMS = [((4, 4, 4, 4), 0.3, 0.120, 2), ((6, 4, 4, 6), 0.4, 0.130, 3), ((4, 4, 4, 8), 0.4, 0.125, 1),
           ((4, 6, 8, 12), 0.4, 0.128, 4)]


@pytest.mark.parametrize("tune", [False, True])
def test_batched_solve(tune):
    from oracle.dirac import WilsonClover
    from paper_1609_02652_gb300 import capi

    gpus, ops, bs, xs, refs, opk = [], [], [], [], [], []
    try:
        for k, (dims, eps, kappa, R) in enumerate(SYSTEMS):
            lat, U = oracle_gauge(dims, eps, 40 + k)
            g = Gpu(lat, U)
            gpus.append(g)
            op = g.op(kappa, 1.0)
            ops.append(op)
            for r in range(R):
                b = lat.even * torch.tensor(pin.spinor(dims, 500 + 10 * k + r)).reshape(*lat.shape, 4, 3)
                bs.append(g.pack(b, 0, 0))
                xs.append(g.buf(0))
                refs.append((g, lat, WilsonClover(lat, U, kappa, 1.0), b, op))
        B = capi.pfmp_batch_create(ops, [s[3] for s in SYSTEMS])
        try:
            if tune:
                block, ms = capi.pfmp_batch_tune(B, 4)
                assert block in (64, 128, 256) and ms > 0
            prm = capi.SolverParams(method=1, tol=1e-10, max_iter=3000, delta=1e-3, check_every=4)
            infos = capi.pfmp_batch_solve(B, prm, xs, bs)
        finally:
            capi.pfmp_batch_destroy(B)
        torch.cuda.synchronize()
        for i, (g, lat, W, b, op) in enumerate(refs):
            x = lat.even * g.unpack(xs[i], 0, 0)
            res = float(torch.linalg.vector_norm(b - W.K(x)) / torch.linalg.vector_norm(b))
            assert res < 1e-10, (i, res)
            assert infos[i].status == 0 and infos[i].true_rel_res < 1e-10
            # the single-system solver on the same rhs
            x1 = g.buf(0)
            capi.pfmp_solve(op, capi.SolverParams(method=0, tol=1e-11, max_iter=3000, delta=0.1, check_every=8), x1,
                            bs[i])
            assert rel_l2(x, lat.even * g.unpack(x1, 0, 0)) < 1e-8
    finally:
        for g in gpus:
            g.close()


def _small_batch(capi, dims=(4, 4, 4, 4), R=2):
    lat, U = oracle_gauge(dims, 0.3, 77)
    g = Gpu(lat, U)
    op = g.op(0.120, 1.0)
    bs = [g.pack(lat.even * torch.tensor(pin.spinor(dims, 900 + r)).reshape(*lat.shape, 4, 3), 0, 0)
          for r in range(R)]
    xs = [g.buf(0) for _ in range(R)]
    return g, op, bs, xs


def test_barrier_wait_is_bounded():
    """The persistent solver's grid barrier: with one block more expected than launched,
    every wait runs out after its limit and the launch returns PFMP_E_TIMEOUT; the context
    stays usable and a batched solve afterwards converges."""
    import time

    from paper_1609_02652_gb300 import capi

    g, op, bs, xs = _small_batch(capi)
    try:
        B = capi.pfmp_batch_create([op], [len(bs)])
        try:
            assert capi.pfmp_batch_barrier_check(B, 64, 0, 2.0) == capi.PFMP_OK
            t0 = time.monotonic()
            st = capi.pfmp_batch_barrier_check(B, 3, 1, 0.5)
            dt = time.monotonic() - t0
            assert st == capi.PFMP_E_TIMEOUT, st
            assert 0.4 < dt < 10.0, dt
            prm = capi.SolverParams(method=1, tol=1e-10, max_iter=3000, delta=1e-3, check_every=4)
            infos = capi.pfmp_batch_solve(B, prm, xs, bs)
            assert all(i.status == 0 and i.true_rel_res < 1e-10 for i in infos)
        finally:
            capi.pfmp_batch_destroy(B)
    finally:
        g.close()


def test_batched_nan_rhs():
    """A right-hand side with a NaN ends the batched solve with PFMP_E_NAN."""
    from paper_1609_02652_gb300 import capi

    g, op, bs, xs = _small_batch(capi)
    try:
        bs[1][5] = float("nan")
        B = capi.pfmp_batch_create([op], [len(bs)])
        try:
            prm = capi.SolverParams(method=1, tol=1e-10, max_iter=3000, delta=1e-3, check_every=4)
            with pytest.raises(capi.PfmpError) as e:
                capi.pfmp_batch_solve(B, prm, xs, bs)
            assert e.value.status == capi.PFMP_E_NAN
        finally:
            capi.pfmp_batch_destroy(B)
    finally:
        g.close()
