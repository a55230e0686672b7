"""GPU parity at the benchmark sizes.

* 16^3 x 32 (the solver benchmark system: eps = 0.5, c_sw = 1.0, kappa = 0.130): K in
  FP64, FP32 and FP16 storage against the oracle's K element by element, in the launch
  configuration the bench uses (the operator's defaults).
* 32^3 x 64 (the stencil roofline lattice; too large for the oracle's whole-lattice K):
  a closed form.  On a pure-gauge field U_mu(x) = g(x) g(x+mu)^dag the operator is the
  free one rotated by g, and a plane wave e^{ipx} chi (p_t antiperiodic) restricted to
  even sites is mapped by M-hat to e^{ipx} M-hat(p) chi with
  M-hat(p) = 1 - 4 kappa^2 (C - i g.s)^2, C = sum_mu cos p_mu, g.s = sum_mu gamma_mu sin p_mu
  (every neighbour of an odd site is even and vice versa).  So K (g psi) = g K(p) psi with
  K(p) = M-hat(p)^dag M-hat(p), checked element by element on all 1,048,576 even sites
  (every link and every boundary of the lattice takes part).
* kappa = 0.134 at 16^3 x 32 (the lightest kappa of the solver scan): the mixed and
  FP16-storage solvers stop on an FP64 true residual below 1e-10, which the oracle's K
  confirms on their solutions.
"""
import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, canon, oracle_gauge, rel_l2

pytestmark = pytest.mark.gpu

BARS = {0: 1e-13, 1: 1e-6, 3: 7.8e-3}


@pytest.fixture(scope="module")
def bench_system():
    from oracle.dirac import WilsonClover

    lat, U = oracle_gauge((16, 16, 16, 32), 0.5, 1)
    g = Gpu(lat, U)
    W = WilsonClover(lat, U, 0.130, 1.0)
    yield lat, U, g, W
    g.close()


@pytest.mark.parametrize("prec", [0, 1, 3], ids=["f64", "f32", "h16"])
def test_K_elementwise_at_16x16x16x32(bench_system, prec):
    from paper_1609_02652_gb300 import capi

    lat, U, g, W = bench_system
    op = g.op(0.130, 1.0)
    psi = lat.even * torch.tensor(pin.spinor(lat.dims, 100)).reshape(*lat.shape, 4, 3)
    ref = W.K(psi)
    b_in, b_out = g.pack(psi, prec, 0), g.buf(prec)
    nrm = capi.pfmp_kop(op, prec, b_out, b_in, want_norm=True)
    got = lat.even * g.unpack(b_out, prec, 0)
    assert rel_l2(got, ref) < BARS[prec]
    assert abs(nrm - (psi.conj() * ref).sum().real.item()) < 10 * BARS[prec] * nrm
    for dagger, r in ((0, W.mhat(psi)), (1, W.mhat_dag(psi))):
        capi.pfmp_mhat(op, prec, b_out, b_in, dagger)
        assert rel_l2(lat.even * g.unpack(b_out, prec, 0), r) < BARS[prec]


def _gammas():
    from oracle.lattice import gammas

    G, _ = gammas()
    return [G[mu].numpy() for mu in range(4)]


def test_K_closed_form_at_32x32x32x64():
    from paper_1609_02652_gb300 import capi

    dims = (32, 32, 32, 64)
    L = np.array(dims)
    V = int(np.prod(L))
    kappa, csw = 0.125, 1.0
    ctx = capi.pfmp_ctx_create(dims, -1, None)
    try:
        # a random SU(3) field g(x): the x-links of exp(i H) from the library's field init
        capi.pfmp_gauge_from_algebra(ctx, np.ascontiguousarray(pin.gauge_algebra(dims, 3)).reshape(-1), 1.0,
                                     capi.PFMP_HOST)
        Ug = np.zeros(V * 72)
        capi.pfmp_gauge_get(ctx, Ug, capi.PFMP_HOST)
        gx = Ug.view(np.complex128).reshape(dims[3], dims[2], dims[1], dims[0], 4, 3, 3)[..., 0, :, :].copy()
        del Ug
        # pure gauge U_mu(x) = g(x) g(x + mu)^dag (axis of mu in (t, z, y, x) order: 3 - mu)
        U = np.empty(gx.shape[:4] + (4, 3, 3), dtype=np.complex128)
        for mu in range(4):
            gn = np.roll(gx, -1, axis=3 - mu)
            U[..., mu, :, :] = np.einsum("...ab,...cb->...ac", gx, gn.conj())
        capi.pfmp_gauge_set(ctx, U.reshape(-1).view(np.float64), capi.PFMP_HOST)
        del U
        op = capi.pfmp_op_create(ctx, kappa, csw)
        # two plane waves with generic spinors, even sites only
        G = _gammas()
        t, z, y, x = np.meshgrid(*[np.arange(n) for n in dims[::-1]], indexing="ij")
        coords = [x, y, z, t]
        even = ((x + y + z + t) % 2 == 0)
        chis = pin.spinor((1, 1, 1, 2), 17).reshape(2, 4, 3)
        psi = np.zeros(gx.shape[:4] + (4, 3), dtype=np.complex128)
        Kpsi = np.zeros_like(psi)
        for w, nvec in enumerate(((1, 2, 3, 4), (5, 0, 7, 11))):
            p = [2 * np.pi * nvec[m] / L[m] for m in range(3)] + [(2 * nvec[3] + 1) * np.pi / L[3]]
            C = sum(np.cos(pm) for pm in p)
            gs = sum(G[m] * np.sin(p[m]) for m in range(4))
            D = C * np.eye(4) - 1j * gs
            Mp = np.eye(4) - 4 * kappa ** 2 * D @ D
            Kp = Mp.conj().T @ Mp
            phase = np.exp(1j * sum(p[m] * coords[m] for m in range(4)))
            psi += phase[..., None, None] * chis[w][None, None, None, None]
            Kpsi += phase[..., None, None] * (Kp @ chis[w])[None, None, None, None]
        psi *= even[..., None, None]
        Kpsi *= even[..., None, None]
        # rotate by g: psi'(x) = g(x) psi(x) (colour index), expected K psi' = g K psi
        psi_g = np.einsum("...ab,...sb->...sa", gx, psi)
        want = np.einsum("...ab,...sb->...sa", gx, Kpsi)
        del psi, Kpsi
        for prec in (0, 1, 3):
            nb = capi.pfmp_spinor_bytes(ctx, prec)
            a = torch.zeros(nb // 4, dtype=torch.float32, device="cuda")
            b = torch.zeros_like(a)
            capi.pfmp_spinor_pack(ctx, a, prec, psi_g.reshape(-1).view(np.float64), capi.PFMP_HOST, 0)
            capi.pfmp_kop(op, prec, b, a)
            out = np.zeros(V * 24)
            capi.pfmp_spinor_unpack(ctx, out, capi.PFMP_HOST, b, prec, 0)
            got = out.view(np.complex128).reshape(want.shape)
            err = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert err < BARS[prec], (prec, err)
        capi.pfmp_op_destroy(op)
    finally:
        capi.pfmp_ctx_destroy(ctx)


@pytest.mark.parametrize("method", [1, 2], ids=["mixed", "half"])
def test_near_critical_kappa_fp64_residual(method):
    from oracle.dirac import WilsonClover
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge((16, 16, 16, 32), 0.5, 1)
    g = Gpu(lat, U)
    try:
        op = g.op(0.134, 1.0)
        b = lat.even * torch.tensor(pin.spinor(lat.dims, 100)).reshape(*lat.shape, 4, 3)
        bb, xx = g.pack(b, 0, 0), g.buf(0)
        prm = capi.SolverParams(method=method, tol=1e-10, max_iter=20000, delta=0.1, check_every=8)
        info = capi.pfmp_solve(op, prm, xx, bb)
        assert info.true_rel_res < 1e-10
        r64 = g.buf(0)
        rel64 = capi.pfmp_true_residual(op, capi.PFMP_F64, r64, xx, bb)
        assert rel64 < 1e-10 and abs(rel64 - info.true_rel_res) < 1e-3 * rel64
        W = WilsonClover(lat, U, 0.134, 1.0)
        x = lat.even * g.unpack(xx, 0, 0)
        res = float(torch.linalg.vector_norm(b - W.K(x)) / torch.linalg.vector_norm(b))
        assert res < 1e-10, res
    finally:
        g.close()
