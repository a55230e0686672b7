"""GPU parity of the field initialisation, Wilson hop, clover term, M-hat and K against
the oracle, element by element, through the C-ABI.  Bars: FP64 relative L2 <= 1e-13,
FP32 <= 1e-6 (the FP32 kernels store links, clover blocks and spinors in FP32 and
accumulate in FP32, so their error is a few ulps of FP32 times the stencil's 8-16
terms)."""
import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, canon, from_canon, oracle_gauge, rel_l2

pytestmark = pytest.mark.gpu

F64_BAR, F32_BAR = 1e-13, 1e-6
# FP16 storage (unit roundoff u = 2^-11): spinors to u of their site's largest component,
# links and clover entries (|.| <= O(1)) to u absolutely, FP32 arithmetic.  One hop sums
# 8 products of a rounded link and a rounded spinor (~2u each, random signs) and rounds
# the output (u): ~4u of its norm; K chains four stencil passes with FP16 intermediates
# and the clover blocks, ~16u.  Bar: 16u = 7.8e-3 for every FP16 result.
H16_BAR = 7.8e-3
BARS = {0: F64_BAR, 1: F32_BAR, 3: H16_BAR}
# several thread blocks and a ragged tail (Vh = 288, 512, 1152 with 128-thread blocks)
LATTICES = [(6, 4, 4, 6), (4, 4, 4, 8), (4, 6, 8, 12)]


@pytest.fixture(scope="module", params=LATTICES, ids=lambda d: "x".join(map(str, d)))
def setup(request):
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(request.param, 0.4, 11)
    g = Gpu(lat, U)
    yield lat, U, g, capi
    g.close()


def spinor(lat, seed):
    return torch.tensor(pin.spinor(lat.dims, seed)).reshape(*lat.shape, 4, 3)


def test_gauge_roundtrip_and_exp(setup):
    lat, U, g, capi = setup
    out = np.zeros(lat.V * 72)
    capi.pfmp_gauge_get(g.ctx, out, capi.PFMP_HOST)
    assert np.array_equal(out, canon(U))
    # field initialisation on the GPU: U = exp(i eps H) from the same coefficients
    from paper_1609_02652_gb300 import capi as c2
    ctx = c2.pfmp_ctx_create(lat.dims, -1)
    try:
        h = np.ascontiguousarray(pin.gauge_algebra(lat.dims, 11)).reshape(-1)
        c2.pfmp_gauge_from_algebra(ctx, h, 0.4, c2.PFMP_HOST)
        got = np.zeros(lat.V * 72)
        c2.pfmp_gauge_get(ctx, got, c2.PFMP_HOST)
        assert np.abs(got - canon(U)).max() < 1e-13
    finally:
        c2.pfmp_ctx_destroy(ctx)


def test_plaquette(setup):
    from oracle.action import mean_plaquette

    lat, U, g, capi = setup
    assert abs(capi.pfmp_plaquette(g.ctx) - mean_plaquette(lat, U)) < 1e-14


@pytest.mark.parametrize("prec", [0, 1, 3], ids=["f64", "f32", "h16"])
@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("parity", [0, 1])
def test_hop(setup, prec, dagger, parity):
    from oracle.dirac import hop

    lat, U, g, capi = setup
    psi = spinor(lat, 3)
    src = lat.mask(1 - parity) * psi
    ref = lat.mask(parity) * hop(lat, U, src, adjoint=bool(dagger))
    op = g.op(0.12, 1.0)
    b_in = g.pack(psi, prec, 1 - parity)
    b_out = g.buf(prec)
    capi.pfmp_dslash(op, prec, b_out, b_in, parity, dagger)
    got = lat.mask(parity) * g.unpack(b_out, prec, parity)
    assert rel_l2(got, ref) < BARS[prec], rel_l2(got, ref)


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
def test_clover_blocks(setup, prec):
    from oracle.dirac import WilsonClover, apply_site_matrix

    lat, U, g, capi = setup
    kappa, csw = 0.125, 1.3
    W = WilsonClover(lat, U, kappa, csw)
    op = g.op(kappa, csw)
    psi = spinor(lat, 4)
    for parity, inverse, A in [(0, 0, W.A), (1, 1, W.Ainv)]:
        ref = lat.mask(parity) * apply_site_matrix(A, psi)
        b_in = g.pack(psi, prec, parity)
        b_out = g.buf(prec)
        capi.pfmp_clover_apply(op, prec, b_out, b_in, parity, inverse)
        got = lat.mask(parity) * g.unpack(b_out, prec, parity)
        assert rel_l2(got, ref) < (F64_BAR if prec == 0 else F32_BAR)
    assert abs(capi.pfmp_op_logdet(op) - W.logdet_oo().item()) < 1e-11 * lat.V


@pytest.mark.parametrize("prec", [0, 1, 3], ids=["f64", "f32", "h16"])
def test_mhat_and_K(setup, prec):
    from oracle.dirac import WilsonClover

    lat, U, g, capi = setup
    kappa, csw = 0.125, 1.0
    W = WilsonClover(lat, U, kappa, csw)
    op = g.op(kappa, csw)
    psi = lat.even * spinor(lat, 5)
    bar = BARS[prec]
    b_in = g.pack(psi, prec, 0)
    b_out = g.buf(prec)
    for dagger, ref in [(0, W.mhat(psi)), (1, W.mhat_dag(psi))]:
        capi.pfmp_mhat(op, prec, b_out, b_in, dagger)
        assert rel_l2(lat.even * g.unpack(b_out, prec, 0), ref) < bar
    nrm = capi.pfmp_kop(op, prec, b_out, b_in, want_norm=True)
    ref = W.K(psi)
    assert rel_l2(lat.even * g.unpack(b_out, prec, 0), ref) < bar
    assert abs(nrm - (psi.conj() * ref).sum().real.item()) < bar * 10 * nrm


def test_blas(setup):
    lat, U, g, capi = setup
    a, b = spinor(lat, 6), spinor(lat, 7)
    for prec in (0, 1):
        x, y = g.pack(a, prec, 0), g.pack(b, prec, 0)
        ae, be = lat.even * a, lat.even * b
        tol = 1e-13 if prec == 0 else 1e-6
        assert abs(capi.pfmp_norm2(g.ctx, prec, x) - (ae.abs() ** 2).sum().item()) < tol * lat.V
        d = capi.pfmp_cdot(g.ctx, prec, x, y)
        assert abs(d - (ae.conj() * be).sum().item()) < tol * lat.V
        capi.pfmp_axpy(g.ctx, prec, 0.3 - 0.7j, x, y)
        assert rel_l2(lat.even * g.unpack(y, prec, 0), be + (0.3 - 0.7j) * ae) < tol
    x64 = g.pack(a, 0, 0)
    x32 = g.buf(1)
    capi.pfmp_convert(g.ctx, x32, 1, x64, 0)
    assert rel_l2(lat.even * g.unpack(x32, 1, 0), lat.even * a) < 1e-7


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("ns", [1, 2, 4, 8])
def test_split_site_kernels(setup, prec, ns):
    """Every threads-per-site variant of the stencil gives M-hat, M-hat^dag, K and the plain
    hop to the parity bar."""
    from oracle.dirac import WilsonClover, hop

    lat, U, g, capi = setup
    W = WilsonClover(lat, U, 0.125, 1.0)
    op = g.op(0.125, 1.0)
    capi.pfmp_op_set_split(op, prec, ns)
    assert capi.pfmp_op_get_split(op, prec) == ns
    bar = F64_BAR if prec == 0 else F32_BAR
    psi = lat.even * spinor(lat, 9)
    bi, bo = g.pack(psi, prec, 0), g.buf(prec)
    for dagger, ref in [(0, W.mhat(psi)), (1, W.mhat_dag(psi))]:
        capi.pfmp_mhat(op, prec, bo, bi, dagger)
        assert rel_l2(lat.even * g.unpack(bo, prec, 0), ref) < bar
    nrm = capi.pfmp_kop(op, prec, bo, bi, want_norm=True)
    ref = W.K(psi)
    assert rel_l2(lat.even * g.unpack(bo, prec, 0), ref) < bar
    assert abs(nrm - (psi.conj() * ref).sum().real.item()) < bar * 10 * nrm
    bo1 = g.buf(prec)
    capi.pfmp_dslash(op, prec, bo1, bi, 1, 0)
    assert rel_l2(lat.odd * g.unpack(bo1, prec, 1), lat.odd * hop(lat, U, psi)) < bar


def test_h16_storage_roundtrip(setup):
    """FP16 spinor storage keeps every component to u = 2^-11 of its site's largest
    |component| (round to nearest: u/2 plus the scale's own rounding), and converts
    to and from FP32 through the library."""
    lat, U, g, capi = setup
    psi = lat.even * spinor(lat, 12)
    h = g.pack(psi, 3, 0)
    back = lat.even * g.unpack(h, 3, 0)
    site_max = torch.view_as_real(psi).abs().amax(dim=(-1, -2, -3))
    err = torch.view_as_real(back - psi).abs().amax(dim=(-1, -2, -3))
    assert float((err / site_max.clamp_min(1e-30))[site_max > 0].max()) <= 2.0 ** -11
    f = g.buf(1)
    capi.pfmp_convert(g.ctx, f, 1, h, 3)
    assert rel_l2(lat.even * g.unpack(f, 1, 0), back) < 1e-7
    h2 = g.buf(3)
    capi.pfmp_convert(g.ctx, h2, 3, f, 1)
    assert rel_l2(lat.even * g.unpack(h2, 3, 0), back) < 1e-7
