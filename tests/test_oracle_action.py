"""Pins of the oracle's PF-MP action terms, heatbath and forces (App. C) against finite
differences of the action, exact heatbath identities and determinant identities."""
import math

import pytest
import torch

import pfmp_inputs as pin
from oracle import cheby
from oracle.action import PFMP, PFMPParams, gauge_action
from oracle.dirac import WilsonClover, dense
from oracle.lattice import C128, F64, Lattice, algebra_to_matrix, expi_hermitian

LINKS = [((1, 2, 3, 0), 2, 5), ((0, 0, 0, 0), 3, 0), ((3, 1, 0, 2), 0, 7), ((2, 3, 1, 1), 1, 2)]


@pytest.fixture(scope="module")
def setup():
    lat = Lattice((4, 4, 4, 4), bc_t=-1)
    h = torch.tensor(pin.gauge_algebra(lat.dims, 1)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), 0.3)
    act = PFMP(lat, PFMPParams(beta=5.5, kappa=0.12, kappa_h=0.11, csw=1.0, n=8))
    xi = [torch.tensor(pin.spinor(lat.dims, 10 + i)).reshape(*lat.shape, 4, 3) * lat.even for i in range(3)]
    phis = act.heatbath(U, *xi)
    return lat, U, act, xi, phis


def _perturbed(U, site, mu, a, e):
    V = U.clone()
    h = torch.zeros(8, dtype=F64)
    h[a] = e
    V[site][mu] = expi_hermitian(algebra_to_matrix(h), 1.0) @ U[site][mu]
    return V


def _fd(S, U, site, mu, a, d=1e-4):
    """Fourth-order central difference of S along U -> exp(i e T_a) U at one link."""
    f = lambda e: float(S(_perturbed(U, site, mu, a, e)))
    return (8 * (f(d) - f(-d)) - (f(2 * d) - f(-2 * d))) / (12 * d)


def test_heatbath_identities(setup):
    """S_i(phi_i) = xi_i^dag xi_i exactly, and R(J) phi_1 = xi_1."""
    lat, U, act, xi, phis = setup
    for i, S in enumerate([act.S_poly, act.S_polycorr, act.S_hasen]):
        s = S(U, phis[i]).item()
        ref = (xi[i].abs() ** 2).sum().item()
        assert abs(s - ref) < 1e-10 * ref
    _, W = act.ops(U)
    p = act.p
    back = cheby.apply_R(W.K, phis[0], p.n, p.mu, p.nu)
    assert (back - xi[0]).abs().max() < 1e-10


@pytest.mark.parametrize("term", ["gauge", "det", "poly", "polycorr", "hasen"])
def test_force_against_finite_difference(setup, term):
    lat, U, act, xi, phis = setup
    S = {
        "gauge": act.S_gauge, "det": act.S_det,
        "poly": lambda V: act.S_poly(V, phis[0]),
        "polycorr": lambda V: act.S_polycorr(V, phis[1]),
        "hasen": lambda V: act.S_hasen(V, phis[2]),
    }[term]
    F = {
        "gauge": act.F_gauge, "det": act.F_det,
        "poly": lambda V: act.F_poly(V, phis[0]),
        "polycorr": lambda V: act.F_polycorr(V, phis[1]),
        "hasen": lambda V: act.F_hasen(V, phis[2]),
    }[term](U)
    scale = F.abs().max().item()
    for site, mu, a in LINKS:
        fd = _fd(S, U, site, mu, a)
        assert abs(F[site][mu][a].item() - fd) < 1e-7 * scale, (term, site, mu, a)


def test_hasenbusch_degenerate_limit():
    """kappa' = kappa: W = M-hat, S_3 = phi^dag phi and F_3 = 0."""
    lat = Lattice((4, 4, 4, 4), bc_t=-1)
    h = torch.tensor(pin.gauge_algebra(lat.dims, 2)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), 0.3)
    act = PFMP(lat, PFMPParams(kappa=0.12, kappa_h=0.12, csw=1.0, n=4))
    phi = torch.tensor(pin.spinor(lat.dims, 3)).reshape(*lat.shape, 4, 3) * lat.even
    s = act.S_hasen(U, phi).item()
    assert abs(s - (phi.abs() ** 2).sum().item()) < 1e-10 * s
    F = act.F_hasen(U, phi)
    assert F.abs().max() < 1e-9


def test_filter_determinant_identity_2x4():
    """det P(J)^{-1} det(J P(J)) det(W K^{-1} W^dag)^{-1} = det K (Sec. 2.2, eq. filter),
    each factor taken by brute force on a dense 2^4 operator."""
    lat = Lattice((2, 2, 2, 2), bc_t=-1)
    h = torch.tensor(pin.gauge_algebra(lat.dims, 4)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), 0.5)
    p = PFMPParams(kappa=0.125, kappa_h=0.11, csw=1.2, n=8)
    M = WilsonClover(lat, U, p.kappa, p.csw)
    W = WilsonClover(lat, U, p.kappa_h, p.csw)
    K, J = dense(lat, M.K), dense(lat, W.K)
    Wd = dense(lat, W.mhat)
    I = torch.eye(K.shape[0], dtype=C128)
    PJ = cheby.norm(p.n, p.mu, p.nu) * I
    for z in cheby.roots(p.n, p.mu, p.nu):
        PJ = PJ @ (J - z * I)
    ld = lambda X: torch.linalg.slogdet(X)[1]
    S3op = Wd @ torch.linalg.solve(K, Wd.conj().T)
    total = -ld(PJ) + ld(J @ PJ) - ld(S3op)
    assert abs(total - ld(K)) < 1e-9


def test_gauge_action_unit_field():
    lat = Lattice((4, 4, 4, 4))
    U = torch.eye(3, dtype=C128).expand(*lat.shape, 4, 3, 3).clone()
    assert abs(gauge_action(lat, U, 5.5).item()) < 1e-12
    # a constant abelian field exp(i theta lambda_3) on x-links only leaves every
    # plaquette trivial (links commute and cancel)
    V = U.clone()
    V[..., 0, :, :] = expi_hermitian(algebra_to_matrix(torch.tensor([0, 0, 1.0, 0, 0, 0, 0, 0], dtype=F64)), 0.8)
    assert abs(gauge_action(lat, V, 5.5).item()) < 1e-11
