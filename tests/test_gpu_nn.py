"""The learned gauge-covariant preconditioner on the GPU: FP64 forward pass and weight
gradients against the oracle's network and its autograd gradients, the FP32 forward
pass, training by the project's own kernels, and FGCR with the trained network against
FGCR without it (the gain) -- every solve judged by the oracle's K at 1e-10."""
import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, canon, oracle_gauge, rel_l2

pytestmark = pytest.mark.gpu

CH = [1, 3, 2, 1]


def _shapes(ch):
    return [(9, co, ci, 4, 4) for ci, co in zip(ch[:-1], ch[1:])]


@pytest.fixture(scope="module")
def world():
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge((4, 4, 4, 8), 0.4, 61)
    g = Gpu(lat, U)
    yield lat, U, g, capi
    g.close()


def test_forward_and_gradient_fp64(world):
    from oracle import nn

    lat, U, g, capi = world
    ws = nn.init_weights(CH, 3)
    net = capi.pfmp_nn_create(g.ctx, CH, capi.PFMP_F64)
    try:
        capi.pfmp_nn_set_weights(net, [w.numpy() for w in ws])
        back = capi.pfmp_nn_get_weights(net, _shapes(CH))
        assert all(np.array_equal(a, w.numpy()) for a, w in zip(back, ws))
        b = lat.even * torch.tensor(pin.spinor(lat.dims, 71)).reshape(*lat.shape, 4, 3)
        x = lat.even * torch.tensor(pin.spinor(lat.dims, 72)).reshape(*lat.shape, 4, 3)
        bb, xx, out = g.pack(b, 0, 0), g.pack(x, 0, 0), g.buf(0)
        capi.pfmp_nn_apply(net, 0, out, bb)
        ref = nn.network_apply(lat, U, ws, b)
        assert rel_l2(lat.even * g.unpack(out, 0, 0), ref) < 1e-12
        L, gr = capi.pfmp_nn_loss_grad(net, bb, xx, _shapes(CH))
        Lo, gro = nn.grads(lat, U, ws, b, x)
        assert abs(L - Lo.item()) < 1e-12 * Lo.item()
        for a, r in zip(gr, gro):
            assert rel_l2(torch.tensor(a), r) < 1e-10
        # the residual loss ||K N(b) - b||^2 / ||b||^2 and its gradient (backward through K)
        from oracle.dirac import WilsonClover

        op = g.op(0.125, 1.0)
        Wop = WilsonClover(lat, U, 0.125, 1.0)
        L, gr = capi.pfmp_nn_loss_grad(net, bb, xx, _shapes(CH), op=op, kind=capi.PFMP_NN_LOSS_RESIDUAL)
        Lo, gro = nn.residual_grads(lat, U, ws, b, Wop.K)
        assert abs(L - Lo.item()) < 1e-12 * Lo.item()
        for a, r in zip(gr, gro):
            assert rel_l2(torch.tensor(a), r) < 1e-10
        # the FP32 instance of the same network
        net32 = capi.pfmp_nn_create(g.ctx, CH, capi.PFMP_F32)
        try:
            capi.pfmp_nn_set_weights(net32, [w.numpy() for w in ws])
            b32, o32 = g.pack(b, 1, 0), g.buf(1)
            capi.pfmp_nn_apply(net32, 1, o32, b32)
            assert rel_l2(lat.even * g.unpack(o32, 1, 0), ref) < 1e-5
        finally:
            capi.pfmp_nn_destroy(net32)
    finally:
        capi.pfmp_nn_destroy(net)


def test_training_and_fgcr_gain(world):
    from oracle.dirac import WilsonClover

    lat, U, g, capi = world
    kappa = 0.128
    op = g.op(kappa, 1.0)
    W = WilsonClover(lat, U, kappa, 1.0)
    mixed = capi.SolverParams(method=1, tol=1e-10, max_iter=4000, delta=1e-4, check_every=8)
    bs, xs = [], []
    for i in range(24):
        b = lat.even * torch.tensor(pin.spinor(lat.dims, 300 + i)).reshape(*lat.shape, 4, 3)
        bb, xx = g.pack(b, 0, 0), g.buf(0)
        capi.pfmp_solve(op, mixed, xx, bb)
        bs.append(bb)
        xs.append(xx)
    ch = [1, 4, 4, 1]
    net = capi.pfmp_nn_create(g.ctx, ch, capi.PFMP_F32)
    try:
        capi.pfmp_nn_set_weights(net, pin.nn_weights(ch, 5))
        R = capi.PFMP_NN_LOSS_RESIDUAL
        l0 = np.mean([capi.pfmp_nn_loss_grad(net, bs[i], xs[i], op=op, kind=R)[0] for i in range(20, 24)])
        capi.pfmp_nn_train(net, bs[:20], xs[:20], steps=800, batch=4, lr=5e-3, op=op, kind=R)
        l1 = np.mean([capi.pfmp_nn_loss_grad(net, bs[i], xs[i], op=op, kind=R)[0] for i in range(20, 24)])  # held out
        assert l1 < 0.75 * l0, (l0, l1)
        prm = capi.SolverParams(method=0, tol=1e-10, max_iter=4000, delta=1e-3, check_every=8, restart=16)
        b = lat.even * torch.tensor(pin.spinor(lat.dims, 999)).reshape(*lat.shape, 4, 3)
        bb = g.pack(b, 0, 0)
        its = {}
        for name, n in [("gcr", None), ("nn", net)]:
            x = g.buf(0)
            info = capi.pfmp_solve_fgcr(op, n, prm, x, bb)
            xo = lat.even * g.unpack(x, 0, 0)
            res = float(torch.linalg.vector_norm(b - W.K(xo)) / torch.linalg.vector_norm(b))
            assert res < 1e-10, (name, res)
            its[name] = info.iters + info.reliable_updates
        print("fgcr iterations", its, "loss", l0, l1)
        assert its["nn"] < its["gcr"], its
    finally:
        capi.pfmp_nn_destroy(net)


CH8 = [1, 8, 8, 8, 1]
# Tensor-core layers take FP16 operands (unit roundoff u = 2^-11) with FP32 accumulation:
# each product carries a relative error of at most 2u, so a layer's output (sums of up
# to 576 such terms that do not cancel) is within about 2u of its norm, and the four
# layers of [1, 8, 8, 8, 1] within 8u = 3.9e-3 of the FP64 network.
TC_BAR = 4e-3


@pytest.mark.parametrize("dims", [(6, 4, 4, 6), (4, 4, 4, 8)], ids=["6x4x4x6_ragged", "4x4x4x8"])
def test_tensor_core_forward(dims):
    """[1, 8, 8, 8, 1]: all four layers on tcgen05 (V = 576 sites is 4.5 tiles of 128: a
    ragged tail) against the oracle's FP64 network; the FP32 kernels alongside;
    a residual 1e-9 times smaller keeps the same relative accuracy (the input is scaled
    by its rms before the FP16 conversion)."""
    from oracle import nn
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(dims, 0.4, 61)
    g = Gpu(lat, U)
    net = capi.pfmp_nn_create(g.ctx, CH8, capi.PFMP_F32)
    try:
        ws = nn.init_weights(CH8, 7)
        capi.pfmp_nn_set_weights(net, [w.numpy() for w in ws])
        b = lat.even * torch.tensor(pin.spinor(lat.dims, 81)).reshape(*lat.shape, 4, 3)
        ref = nn.network_apply(lat, U, ws, b)
        out = g.buf(1)
        capi.pfmp_nn_apply(net, 1, out, g.pack(b, 1, 0))
        err = rel_l2(lat.even * g.unpack(out, 1, 0), ref)
        assert err < TC_BAR, err
        capi.pfmp_nn_apply(net, 1, out, g.pack(1e-9 * b, 1, 0))
        err_small = rel_l2(lat.even * g.unpack(out, 1, 0), 1e-9 * ref)
        assert err_small < TC_BAR, err_small
        capi.pfmp_nn_set_tensor_cores(net, 0)
        capi.pfmp_nn_apply(net, 1, out, g.pack(b, 1, 0))
        assert rel_l2(lat.even * g.unpack(out, 1, 0), ref) < 1e-5
        print("tensor-core network error", err, err_small)
    finally:
        capi.pfmp_nn_destroy(net)
        g.close()


def test_tensor_core_fgcr_converges(world):
    """FGCR with the tensor-core network reaches the 1e-10 true residual (oracle K)."""
    from oracle.dirac import WilsonClover

    lat, U, g, capi = world
    op = g.op(0.125, 1.0)
    W = WilsonClover(lat, U, 0.125, 1.0)
    net = capi.pfmp_nn_create(g.ctx, CH8, capi.PFMP_F32)
    try:
        capi.pfmp_nn_set_weights(net, pin.nn_weights(CH8, 9))
        prm = capi.SolverParams(method=0, tol=1e-10, max_iter=4000, delta=1e-3, check_every=8, restart=16)
        b = lat.even * torch.tensor(pin.spinor(lat.dims, 998)).reshape(*lat.shape, 4, 3)
        x = g.buf(0)
        capi.pfmp_solve_fgcr(op, net, prm, x, g.pack(b, 0, 0))
        xo = lat.even * g.unpack(x, 0, 0)
        res = float(torch.linalg.vector_norm(b - W.K(xo)) / torch.linalg.vector_norm(b))
        assert res < 1e-10, res
    finally:
        capi.pfmp_nn_destroy(net)
