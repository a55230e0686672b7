"""Pins of the oracle's spectral-range functions (App. A): the free-field closed form of
K's eigenvalues, the Lanczos tridiagonal against an explicit orthonormal basis, and
Ritz values that bracket and converge to the dense extremes."""
import math

import numpy as np
import torch

import pfmp_inputs as pin
from oracle.dirac import WilsonClover, dense
from oracle.lattice import C128, Lattice, algebra_to_matrix, expi_hermitian
from oracle.spectrum import extreme_eigenvalues, lanczos, ritz_extremes


def _gauge(lat, eps, seed):
    h = torch.tensor(pin.gauge_algebra(lat.dims, seed)).reshape(*lat.shape, 4, 8)
    return expi_hermitian(algebra_to_matrix(h), eps)


def test_free_field_extremes_closed_form():
    """U = 1: the eigenvalues of K are |1 - 4 kappa^2 (C +- i s)^2|^2 over the momenta
    (antiperiodic in time), C = sum cos p, s^2 = sum sin^2 p."""
    lat = Lattice((2, 2, 2, 4), bc_t=-1)
    U = torch.eye(3, dtype=C128).expand(*lat.shape, 4, 3, 3).clone()
    kappa = 0.11
    vals = []
    for n in np.ndindex(*lat.dims):
        p = [2 * math.pi * n[m] / lat.dims[m] for m in range(4)]
        p[3] += math.pi / lat.dims[3]
        C = sum(math.cos(q) for q in p)
        s = math.sqrt(sum(math.sin(q) ** 2 for q in p))
        for sg in (1, -1):
            vals.append(abs(1 - 4 * kappa ** 2 * (C + sg * 1j * s) ** 2) ** 2)
    lo, hi = extreme_eigenvalues(lat, U, kappa, 1.3)
    assert abs(lo - min(vals)) < 1e-12 and abs(hi - max(vals)) < 1e-12


def test_lanczos_is_a_projection():
    """T_k = Q^dag K Q for the orthonormal Krylov basis Q built by Gram-Schmidt with full
    reorthogonalisation (early steps, where the plain recurrence is still orthogonal)."""
    lat = Lattice((2, 2, 2, 2), bc_t=-1)
    U = _gauge(lat, 0.5, 3)
    op = WilsonClover(lat, U, 0.12, 1.0)
    v0 = lat.even * torch.tensor(pin.spinor(lat.dims, 5)).reshape(*lat.shape, 4, 3)
    k = 8
    a, b = lanczos(op.K, v0, k)
    Kd = dense(lat, op.K)
    from oracle.dirac import to_parity_vector
    q = [to_parity_vector(lat, v0)]
    q[0] = q[0] / torch.linalg.norm(q[0])
    for j in range(k - 1):
        w = Kd @ q[-1]
        for qq in q:
            w = w - (qq.conj() @ w) * qq
        q.append(w / torch.linalg.norm(w))
    Q = torch.stack(q, 1)
    T = Q.conj().T @ Kd @ Q
    assert (T.diagonal().real - a).abs().max() < 1e-12
    assert (T.diagonal(1).abs() - b[:k - 1]).abs().max() < 1e-12


def test_ritz_values_bracket_and_converge():
    lat = Lattice((4, 4, 4, 4), bc_t=-1)
    U = _gauge(lat, 0.3, 1)
    op = WilsonClover(lat, U, 0.12, 1.0)
    lo, hi = extreme_eigenvalues(lat, U, 0.12, 1.0)
    v0 = lat.even * torch.tensor(pin.spinor(lat.dims, 7)).reshape(*lat.shape, 4, 3)
    a, b = lanczos(op.K, v0, 200)
    prev = None
    for k in (10, 40, 200):
        rl, rh = ritz_extremes(a[:k], b[:k])
        assert lo - 1e-12 <= rl and rh <= hi + 1e-12
        if prev:
            assert rl <= prev[0] + 1e-12 and rh >= prev[1] - 1e-12   # interlacing: extremes move outwards
        prev = (rl, rh)
    assert abs(prev[1] - hi) < 1e-10 * hi
    assert abs(prev[0] - lo) < 1e-6 * lo
