"""Pins of the oracle's lattice algebra and Dirac operator against closed forms,
invariants and brute force (none of them re-derives the oracle's own formula)."""
import math

import numpy as np
import pytest
import torch

import pfmp_inputs as pin
from oracle.dirac import WilsonClover, dense, from_parity_vector, gamma5, hop, to_parity_vector
from oracle.lattice import (C128, F64, Lattice, algebra_to_matrix, dagger, expi_hermitian, gammas,
                            matrix_to_algebra, su3_generators)


def random_gauge(lat, eps, seed):
    h = torch.tensor(pin.gauge_algebra(lat.dims, seed)).reshape(*lat.shape, 4, 8)
    return expi_hermitian(algebra_to_matrix(h), eps)


def even_spinor(lat, seed):
    return torch.tensor(pin.spinor(lat.dims, seed)).reshape(*lat.shape, 4, 3) * lat.even


def test_gamma_algebra():
    G, g5 = gammas()
    I = torch.eye(4, dtype=C128)
    for a in range(4):
        assert torch.allclose(G[a], dagger(G[a]))
        for b in range(4):
            ac = G[a] @ G[b] + G[b] @ G[a]
            assert torch.allclose(ac, 2 * I * (a == b))
    assert torch.allclose(g5, torch.diag(torch.tensor([1, 1, -1, -1], dtype=C128)))


def test_su3_generators_and_exp():
    T = su3_generators()
    tr = torch.einsum("aij,bji->ab", T, T)
    assert torch.allclose(tr, 0.5 * torch.eye(8, dtype=C128), atol=1e-15)
    # [T_1, T_2] = i T_3 (structure constant f_123 = 1)
    assert torch.allclose(T[0] @ T[1] - T[1] @ T[0], 1j * T[2], atol=1e-15)
    h = torch.tensor(np.random.default_rng(3).standard_normal((50, 8)))
    assert torch.allclose(matrix_to_algebra(algebra_to_matrix(h)), h, atol=1e-14)
    U = expi_hermitian(algebra_to_matrix(h), 0.7)
    eye = torch.eye(3, dtype=C128)
    assert (U @ dagger(U) - eye).abs().max() < 1e-14
    assert (torch.linalg.det(U) - 1).abs().max() < 1e-14
    # exp(i eps H) against the Taylor series (independent of the eigendecomposition)
    X = 0.7j * algebra_to_matrix(h)
    E, term = eye.expand_as(X).clone(), eye.expand_as(X).clone()
    for k in range(1, 40):
        term = term @ X / k
        E = E + term
    assert (E - U).abs().max() < 1e-13


def _free_spectrum(lat, kappa, antiperiodic):
    vals = []
    L = lat.dims
    for n in np.ndindex(*L):
        p = [2 * math.pi * n[m] / L[m] for m in range(4)]
        if antiperiodic:
            p[3] += math.pi / L[3]
        Cc = sum(math.cos(q) for q in p)
        s = math.sqrt(sum(math.sin(q) ** 2 for q in p))
        for sg in (1, -1):
            vals += [1 - 4 * kappa ** 2 * (Cc + sg * 1j * s) ** 2] * 3
    return np.array(vals)


def _match_multisets(a, b, tol):
    a = list(a)
    b = list(b)
    assert len(a) == len(b)
    used = np.zeros(len(b), bool)
    bb = np.array(b)
    for x in a:
        d = np.abs(bb - x) + used * 1e9
        j = int(np.argmin(d))
        assert d[j] < tol, (x, bb[j])
        used[j] = True


@pytest.mark.parametrize("bc", [-1, 1])
def test_free_field_spectrum_closed_form(bc):
    """U = 1: eigenvalues of M-hat are 1 - 4 kappa^2 (C +- i s)^2 (momentum space)."""
    lat = Lattice((4, 4, 4, 4), bc_t=bc)
    U = torch.eye(3, dtype=C128).expand(*lat.shape, 4, 3, 3).clone()
    kappa = 0.13
    op = WilsonClover(lat, U, kappa, 1.7)       # clover vanishes on the free field
    assert (op.A - torch.eye(12, dtype=C128)).abs().max() < 1e-15
    ev = torch.linalg.eigvals(dense(lat, op.mhat)).numpy()
    _match_multisets(ev, _free_spectrum(lat, kappa, bc == -1), 1e-10)


def test_forward_hop_convention():
    """A point source at y feeds x = y - mu with (1 - gamma_mu) U_mu(x) and x = y + mu with
    (1 + gamma_mu) U_mu(y)^dag; across the time boundary with the factor bc_t."""
    lat = Lattice((4, 4, 4, 4), bc_t=-1)
    U = random_gauge(lat, 0.4, 2)
    G, _ = gammas()
    psi = torch.zeros(*lat.shape, 4, 3, dtype=C128)
    v = torch.tensor(pin.spinor((1, 1, 1, 1), 4)).reshape(4, 3)
    y = (0, 1, 2, 3)          # (t, z, y, x) index: t = 0 boundary slab
    psi[y] = v
    out = hop(lat, U, psi)
    # x = y - t-hat wraps to t = Lt - 1: forward hop across the boundary, factor -1
    xm = (3, 1, 2, 3)
    Uv = (U[xm][3] @ v.T).T
    expect = -(torch.eye(4, dtype=C128) - G[3]) @ Uv
    assert torch.allclose(out[xm], expect, atol=1e-14)
    xp = (0, 1, 2, 0)          # y + x-hat (x wraps 3 -> 0): backward hop from x
    Uv = (dagger(U[y][0]) @ v.T).T
    expect = (torch.eye(4, dtype=C128) + G[0]) @ Uv
    assert torch.allclose(out[xp], expect, atol=1e-14)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4)])
def test_adjoint_and_gamma5_hermiticity_dense(dims):
    lat = Lattice(dims, bc_t=-1)
    U = random_gauge(lat, 0.5, 7)
    op = WilsonClover(lat, U, 0.125, 1.3)
    D = dense(lat, op.mhat)
    Dd = dense(lat, op.mhat_dag)
    assert (Dd - D.conj().T).abs().max() < 1e-14
    n = D.shape[0]
    g5 = torch.diag(torch.tensor([1, 1, -1, -1], dtype=C128))
    G5 = torch.kron(torch.eye(n // 12, dtype=C128), torch.kron(g5, torch.eye(3, dtype=C128)))
    assert (G5 @ D @ G5 - D.conj().T).abs().max() < 1e-14
    K = dense(lat, op.K)
    assert torch.linalg.eigvalsh(K).min() > 0


def test_gamma5_hermiticity_4x4x4x8():
    lat = Lattice((4, 4, 4, 8), bc_t=-1)
    U = random_gauge(lat, 0.3, 1)
    op = WilsonClover(lat, U, 0.12, 1.0)
    u, v = even_spinor(lat, 1), even_spinor(lat, 2)
    lhs = (u.conj() * op.mhat(v)).sum()
    rhs = (gamma5(op.mhat(gamma5(u))).conj() * v).sum()
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    lhs = (u.conj() * op.mhat(v)).sum()
    rhs = (op.mhat_dag(u).conj() * v).sum()
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_clover_hermitian_chiral_blocks():
    lat = Lattice((4, 4, 4, 4))
    U = random_gauge(lat, 0.5, 3)
    op = WilsonClover(lat, U, 0.13, 1.6)
    A = op.A
    assert (A - dagger(A)).abs().max() < 1e-15
    # sigma_{mu nu} commutes with gamma_5: no coupling between spins {0,1} and {2,3}
    assert A[..., :6, 6:].abs().max() < 1e-15
    assert (A - torch.eye(12, dtype=C128)).abs().max() > 1e-3


def test_gauge_covariance():
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^dag, psi -> g psi gives M-hat -> g M-hat g^dag."""
    lat = Lattice((4, 4, 4, 4), bc_t=-1)
    U = random_gauge(lat, 0.4, 5)
    g = random_gauge(lat, 1.0, 6)[..., 0, :, :]
    Ug = torch.stack([g @ U[..., mu, :, :] @ dagger(lat.fwd(g, mu)) for mu in range(4)], dim=-3)
    psi = even_spinor(lat, 3)
    gpsi = torch.einsum("tzyxab,tzyxsb->tzyxsa", g, psi)
    K, Kg = WilsonClover(lat, U, 0.12, 1.0).K, WilsonClover(lat, Ug, 0.12, 1.0).K
    lhs = Kg(gpsi)
    rhs = torch.einsum("tzyxab,tzyxsb->tzyxsa", g, K(psi))
    assert (lhs - rhs).abs().max() < 1e-13
    a = WilsonClover(lat, U, 0.12, 1.0).logdet_oo()
    b = WilsonClover(lat, Ug, 0.12, 1.0).logdet_oo()
    assert abs(a - b) < 1e-12


def test_schur_determinant_identity():
    """det M = det M_oo det M-hat on a 2^4 lattice (full matrix assembled by brute force)."""
    lat = Lattice((2, 2, 2, 2), bc_t=-1)
    U = random_gauge(lat, 0.6, 9)
    op = WilsonClover(lat, U, 0.13, 1.2)
    n = lat.V * 12
    e = torch.eye(n, dtype=C128).reshape(n, *lat.shape, 4, 3)
    Mfull = op.M(e).reshape(n, n).T
    _, ld_full = torch.linalg.slogdet(Mfull)
    _, ld_hat = torch.linalg.slogdet(dense(lat, op.mhat))
    assert abs(ld_full - (ld_hat + op.logdet_oo())) < 1e-11


def test_wilson_limit():
    """c_sw = 0: M-hat = 1 - kappa^2 H_eo H_oe."""
    lat = Lattice((4, 4, 4, 4), bc_t=-1)
    U = random_gauge(lat, 0.4, 8)
    psi = even_spinor(lat, 8)
    kappa = 0.14
    op = WilsonClover(lat, U, kappa, 0.0)
    ref = psi - kappa ** 2 * lat.even * hop(lat, U, lat.odd * hop(lat, U, psi))
    assert (op.mhat(psi) - ref).abs().max() < 1e-14


def test_parity_vector_roundtrip():
    lat = Lattice((4, 4, 4, 8))
    psi = even_spinor(lat, 4)
    v = to_parity_vector(lat, psi, 0)
    assert v.numel() == lat.V // 2 * 12
    assert torch.equal(from_parity_vector(lat, v, 0), psi)
