"""GPU parity of the spectral-range estimate (App. A) against the oracle: the Lanczos
tridiagonal's first coefficients against the oracle's plain recurrence, the extreme
Ritz values against the dense eigenvalues of K at 4^4 and 4x4x4x8, and at 16^3x32
(the benchmark operator) properties that hold at any size: the Ritz extremes move
outwards with the step count, and a Rayleigh quotient lies inside them."""
import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, oracle_gauge

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,kappa", [((4, 4, 4, 4), 0.12), ((4, 4, 4, 8), 0.13)])
def test_extremes_match_dense(dims, kappa):
    from oracle.dirac import WilsonClover
    from oracle.spectrum import extreme_eigenvalues, lanczos
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge(dims, 0.3, 1)
    g = Gpu(lat, U)
    try:
        op = g.op(kappa, 1.0)
        v0 = lat.even * torch.tensor(pin.spinor(dims, 7)).reshape(*lat.shape, 4, 3)
        lo, hi, a, b = capi.pfmp_spectrum(op, 400, g.pack(v0, 0, 0))
        rlo, rhi = extreme_eigenvalues(lat, U, kappa, 1.0)
        assert rlo - 1e-12 <= lo and hi <= rhi + 1e-12
        assert abs(hi - rhi) < 1e-10 * rhi
        assert abs(lo - rlo) < 1e-6 * rlo
        ra, rb = lanczos(WilsonClover(lat, U, kappa, 1.0).K, v0, 12)
        assert np.abs(a[:12] - ra.numpy()).max() < 1e-12 * np.abs(ra.numpy()).max()
        assert np.abs(b[:12] - rb.numpy()).max() < 1e-12 * np.abs(rb.numpy()).max()
    finally:
        g.close()


def test_closed_krylov_space():
    """On 2^4 (96 unknowns per parity) more steps than unknowns end early with the exact
    extremes."""
    from oracle.spectrum import extreme_eigenvalues
    from paper_1609_02652_gb300 import capi

    dims = (2, 2, 2, 2)
    lat, U = oracle_gauge(dims, 0.5, 4)
    g = Gpu(lat, U)
    try:
        v0 = lat.even * torch.tensor(pin.spinor(dims, 3)).reshape(*lat.shape, 4, 3)
        lo, hi, a, _ = capi.pfmp_spectrum(g.op(0.125, 1.2), 300, g.pack(v0, 0, 0))
        rlo, rhi = extreme_eigenvalues(lat, U, 0.125, 1.2)
        assert len(a) <= 300
        assert abs(hi - rhi) < 1e-10 * rhi and abs(lo - rlo) < 1e-8 * rlo
        with pytest.raises(capi.PfmpError):
            capi.pfmp_spectrum(g.op(0.125, 1.2), 10, g.buf(0))   # zero start vector
    finally:
        g.close()


def test_benchmark_operator_properties():
    """16^3x32, eps 0.5, kappa 0.130, c_sw 1: more steps widen the Ritz range, and the
    Rayleigh quotient <v, K v>/<v, v> of the start vector (K through the library, whose
    parity is tested elsewhere) lies inside it."""
    from paper_1609_02652_gb300 import capi

    dims = (16, 16, 16, 32)
    lat, U = oracle_gauge(dims, 0.5, 1)
    g = Gpu(lat, U)
    try:
        op = g.op(0.130, 1.0)
        v0 = lat.even * torch.tensor(pin.spinor(dims, 100)).reshape(*lat.shape, 4, 3)
        b0 = g.pack(v0, 0, 0)
        prev = None
        for k in (20, 100, 400):
            lo, hi, _, _ = capi.pfmp_spectrum(op, k, b0)
            assert 0 < lo < hi
            if prev:
                assert lo <= prev[0] * (1 + 1e-12) and hi >= prev[1] * (1 - 1e-12)
            prev = (lo, hi)
        # Rayleigh quotient of K on random vectors (through the library's own K and dot,
        # whose parity is tested elsewhere) must lie inside [lo, hi]
        x = g.pack(v0, 0, 0)
        y = g.buf(0)
        kk = capi.pfmp_kop(op, 0, y, x, want_norm=True)
        rq = kk / capi.pfmp_norm2(g.ctx, 0, x)
        assert prev[0] <= rq <= prev[1]
    finally:
        g.close()
