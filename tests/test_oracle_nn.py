"""Pins of the oracle's gauge-covariant network: gauge covariance, linearity, the
identity limit, and autograd gradients against finite differences."""
import numpy as np
import torch

import pfmp_inputs as pin
from oracle import nn
from oracle.lattice import C128, Lattice, algebra_to_matrix, dagger, expi_hermitian


def _setup(dims=(4, 4, 4, 4), seed=3):
    lat = Lattice(dims, bc_t=-1)
    h = torch.tensor(pin.gauge_algebra(dims, seed)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), 0.4)
    b = lat.even * torch.tensor(pin.spinor(dims, seed + 1)).reshape(*lat.shape, 4, 3)
    return lat, U, b


def test_gauge_covariance():
    lat, U, b = _setup()
    ws = nn.init_weights([1, 3, 2, 1], 5)
    g = expi_hermitian(algebra_to_matrix(torch.tensor(pin.gauge_algebra(lat.dims, 9)).reshape(*lat.shape, 4, 8)), 1.0)[..., 0, :, :]
    Ug = torch.stack([g @ U[..., mu, :, :] @ dagger(lat.fwd(g, mu)) for mu in range(4)], dim=-3)
    gb = torch.einsum("tzyxab,tzyxsb->tzyxsa", g, b)
    lhs = nn.network_apply(lat, Ug, ws, gb)
    rhs = torch.einsum("tzyxab,tzyxsb->tzyxsa", g, nn.network_apply(lat, U, ws, b))
    assert (lhs - rhs).abs().max() < 1e-13


def test_identity_and_linearity():
    lat, U, b = _setup()
    ws = [torch.zeros(9, 1, 1, 4, 4, dtype=C128)]
    ws[0][0, 0, 0] = torch.eye(4, dtype=C128) * (0.5 - 0.25j)
    assert (nn.network_apply(lat, U, ws, b) - (0.5 - 0.25j) * b).abs().max() < 1e-15
    ws = nn.init_weights([1, 4, 1], 2)
    b2 = lat.even * torch.tensor(pin.spinor(lat.dims, 11)).reshape(*lat.shape, 4, 3)
    a = nn.network_apply(lat, U, ws, 2j * b + b2)
    c = 2j * nn.network_apply(lat, U, ws, b) + nn.network_apply(lat, U, ws, b2)
    assert (a - c).abs().max() < 1e-13


def test_single_hop_matches_wilson_hop():
    """With W_f = (1 - g_mu), W_b = (1 + g_mu) and no site term, one layer is the Wilson hop."""
    from oracle.dirac import hop
    from oracle.lattice import gammas

    lat, U, b = _setup()
    G, _ = gammas()
    I4 = torch.eye(4, dtype=C128)
    W = torch.zeros(9, 1, 1, 4, 4, dtype=C128)
    for mu in range(4):
        W[1 + mu, 0, 0] = I4 - G[mu]
        W[5 + mu, 0, 0] = I4 + G[mu]
    y = nn.layer_apply(lat, U, W, b.unsqueeze(0))[0]
    assert (y - hop(lat, U, b)).abs().max() < 1e-14


def test_gradient_against_finite_differences():
    lat, U, b = _setup((2, 2, 2, 4))
    x = lat.even * torch.tensor(pin.spinor(lat.dims, 13)).reshape(*lat.shape, 4, 3)
    ws = nn.init_weights([1, 2, 1], 7)
    L, gr = nn.grads(lat, U, ws, b, x)
    rng = np.random.default_rng(0)
    for trial in range(6):
        l = trial % 2
        idx = tuple(int(rng.integers(0, n)) for n in ws[l].shape)
        for part in (1.0, 1j):
            d = 1e-6
            wp = [w.clone() for w in ws]
            wm = [w.clone() for w in ws]
            wp[l][idx] += d * part
            wm[l][idx] -= d * part
            fd = (nn.loss(lat, U, wp, b, x) - nn.loss(lat, U, wm, b, x)).item() / (2 * d)
            an = gr[l][idx].real.item() if part == 1.0 else gr[l][idx].imag.item()
            assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (trial, part, fd, an)
