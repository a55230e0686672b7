"""Pins of the oracle's Chebyshev filter (App. A), partial fractions (App. C) and solvers."""
import json
import math
import os

import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from oracle import cheby
from oracle.dirac import WilsonClover, dense, from_parity_vector, to_parity_vector
from oracle.lattice import C128, Lattice, algebra_to_matrix, expi_hermitian
from oracle.solvers import cg, multishift_cg, shifted_solve

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cheb_T(m, x):
    """Chebyshev polynomial of the first kind by its three-term recurrence."""
    a, b = torch.ones_like(x), x
    if m == 0:
        return a
    for _ in range(m - 1):
        a, b = b, 2 * x * b - a
    return b


@pytest.mark.parametrize("n", [2, 4, 8, 12, 48])
def test_normalisation_and_conjugate_pairs(n):
    mu, nu = 1.2, 0.9
    z = cheby.roots(n, mu, nu)
    a = 1.0 / (mu * torch.prod(mu - z))
    assert abs(a.imag) < 1e-12 * abs(a.real) and a.real > 0
    # P(mu) = 1/mu exactly (definition of a_n)
    assert abs(cheby.poly_scalar(torch.tensor(mu, dtype=torch.float64), n, mu, nu) - 1 / mu) < 1e-13
    # roots are real or come in conjugate pairs -> P real on the real axis, positive for even n
    zs = sorted(z.tolist(), key=lambda c: (round(c.real, 12), c.imag))
    zc = sorted(z.conj().tolist(), key=lambda c: (round(c.real, 12), c.imag))
    assert np.allclose(zs, zc, atol=1e-13)
    x = torch.linspace(0.0, 2.6, 301, dtype=torch.float64)
    P = cheby.poly_scalar(x, n, mu, nu)
    assert P.imag.abs().max() < 1e-10 * P.real.abs().max()
    assert (P.real > 0).all()


def test_ellipse_geometry_fig_a1():
    """With the origin added, the n+1 points sit at equal angles 2 pi k/(n+1) on the ellipse
    of semi-axes mu (real) and sqrt(mu^2 - nu^2) centred at mu; Fig. A.1 draws n = 4 at
    +-36 and +-108 degrees."""
    n, mu, nu = 4, 1.2, 0.9
    z = cheby.roots(n, mu, nu)
    b = math.sqrt(mu * mu - nu * nu)
    ang = torch.atan2(z.imag / b, (z.real - mu) / mu) * 180 / math.pi
    got = sorted(float(a) for a in ang)
    assert np.allclose(got, [-108, -36, 36, 108], atol=1e-10)


@pytest.mark.parametrize("n", [4, 8, 12])
def test_closed_form_error(n):
    """1 - z P_n(z) = T_{n+1}((mu - z)/nu) / T_{n+1}(mu/nu), so the largest relative error of
    P_n against 1/x on [mu - nu, mu + nu] is 1 / T_{n+1}(mu/nu)."""
    mu, nu = 1.2, 0.9
    zz = torch.tensor([0.3 + 0.1j, 1.5 - 0.2j, 2.0, 0.01, 0.7 + 0.6j], dtype=C128)
    lhs = 1 - zz * cheby.poly_scalar(zz, n, mu, nu)
    rhs = _cheb_T(n + 1, (mu - zz) / nu) / _cheb_T(n + 1, torch.tensor(mu / nu, dtype=C128))
    assert (lhs - rhs).abs().max() < 1e-11
    x = torch.linspace(mu - nu, mu + nu, 4001, dtype=torch.float64)
    err = (1 - x * cheby.poly_scalar(x, n, mu, nu).real).abs().max().item()
    bound = 1.0 / math.cosh((n + 1) * math.acosh(mu / nu))
    assert abs(err - bound) < 1e-6 * max(bound, 1e-12) + 1e-12


def test_factorisation_rule():
    """P_{p1} divides P_{p2} when (p1 + 1) | (p2 + 1) (App. A): roots of P_4 lie among P_24's."""
    r4 = cheby.roots(4, 1.2, 0.9)
    r24 = cheby.roots(24, 1.2, 0.9)
    for z in r4:
        assert (r24 - z).abs().min() < 1e-13
    r12 = cheby.roots(12, 1.2, 0.9)
    r48 = cheby.roots(48, 1.2, 0.9)     # 13 does not divide 49
    assert min((r48 - z).abs().min().item() for z in r12) > 1e-3


@pytest.mark.parametrize("n", [4, 8, 12])
def test_partial_fractions(n):
    """sum_i r_i / (z - z_i) = 1 / (z P_n(z)) with z_{n+1} = 0 (App. C)."""
    mu, nu = 1.2, 0.9
    shifts, r = cheby.residues(n, mu, nu)
    zz = torch.tensor([0.37 + 0.2j, 1.9, 0.05 - 0.01j, 2.5 + 1j], dtype=C128)
    lhs = (r / (zz[:, None] - shifts)).sum(-1)
    rhs = 1.0 / (zz * cheby.poly_scalar(zz, n, mu, nu))
    assert ((lhs - rhs).abs() / rhs.abs()).max() < 1e-11
    zh, s = cheby.half_residues(n, mu, nu)
    lhs = (s / (zz[:, None] - zh)).sum(-1)
    rhs = 1.0 / torch.prod(zz[:, None] - zh, -1)
    assert ((lhs - rhs).abs() / rhs.abs()).max() < 1e-11
    # R^dag R = P on the real axis
    x = torch.linspace(0.01, 2.5, 50, dtype=torch.float64).to(C128)
    R = math.sqrt(cheby.norm(n, mu, nu)) * torch.prod(x[:, None] - zh, -1)
    assert ((R.conj() * R - cheby.poly_scalar(x, n, mu, nu)).abs()).max() < 1e-12
    with pytest.raises(ValueError):
        cheby.half_roots(5, mu, nu)


def _setup(dims=(2, 2, 2, 2), kappa=0.125, csw=1.0, seed=3):
    lat = Lattice(dims, bc_t=-1)
    h = torch.tensor(pin.gauge_algebra(lat.dims, seed)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), 0.4)
    op = WilsonClover(lat, U, kappa, csw)
    b = torch.tensor(pin.spinor(lat.dims, seed + 1)).reshape(*lat.shape, 4, 3) * lat.even
    return lat, op, b


def test_poly_apply_against_eigendecomposition():
    """P(J) v by the product of roots equals V P(Lambda) V^dag v on a dense 2^4 J, up to
    the orders of the large filters (12, 48, 64).  In the order k = 1..n the partial
    products pass through values far from |P|, so rounding grows with the order: measured
    2e-15 (n <= 12), 2e-13 (48), 4e-12 (64) of max |P v|; the bars allow 5x that."""
    lat, op, b = _setup()
    Jd = dense(lat, op.K)
    lam, V = torch.linalg.eigh(Jd)
    for n, bar in ((4, 1e-14), (8, 1e-14), (12, 1e-14), (48, 1e-12), (64, 2e-11)):
        Plam = cheby.poly_scalar(lam, n, 1.2, 0.9)
        ref = V @ (Plam * (V.conj().T @ to_parity_vector(lat, b)))
        got = to_parity_vector(lat, cheby.apply_poly(op.K, b, n, 1.2, 0.9))
        assert (got - ref).abs().max() < bar * ref.abs().max(), n


def test_cg_against_dense_lu():
    lat, op, b = _setup()
    x, it, res = cg(op.K, b, tol=1e-13)
    assert res < 1e-12
    Kd = dense(lat, op.K)
    ref = torch.linalg.solve(Kd, to_parity_vector(lat, b))
    got = to_parity_vector(lat, x)
    assert (got - ref).abs().max() < 1e-11 * ref.abs().max()


def test_shifted_solves_against_dense():
    lat, op, b = _setup()
    shifts, _ = cheby.residues(8, 1.2, 0.9)
    Kd = dense(lat, op.K)
    bv = to_parity_vector(lat, b)
    x_ms, it = multishift_cg(op.K, b, -shifts, tol=1e-13)
    x_nr, _, res = shifted_solve(op.K, b, shifts, tol=1e-13)
    assert res.max() < 1e-11
    I = torch.eye(Kd.shape[0], dtype=C128)
    for i, z in enumerate(shifts):
        ref = torch.linalg.solve(Kd - z * I, bv)
        for x in (x_ms, x_nr):
            got = to_parity_vector(lat, x[i])
            assert (got - ref).abs().max() < 1e-11 * ref.abs().max()


def test_force_count_table_3_2():
    """The polynomial force needs exactly 2p - 2 applications of K besides dK/dU (Table 3.2)."""
    from oracle.action import PFMP, PFMPParams
    import oracle.dirac as dirac

    with open(os.path.join(GOLDEN, "table32_force_counts.json")) as f:
        gold = json.load(f)
    lat, op, b = _setup()
    counts = []
    orig = dirac.WilsonClover.K
    for p in gold["p"]:
        act = PFMP(lat, PFMPParams(n=p, kappa=0.125, kappa_h=0.125))
        calls = []

        def counting(self, psi, _orig=orig, _calls=calls):
            if not psi.requires_grad and not any(t.requires_grad for t in [self.U]):
                _calls.append(psi.shape[0] if psi.dim() == 7 else 1)
            return _orig(self, psi)

        dirac.WilsonClover.K = counting
        try:
            act.F_poly(op.U, b)
        finally:
            dirac.WilsonClover.K = orig
        counts.append(sum(calls))
    assert counts == gold["mat_per_F1"]
