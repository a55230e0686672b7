"""Pins of the oracle's gauge-covariant network: gauge covariance, linearity, the
identity limit, autograd gradients of both losses against finite differences, and the
residual loss against a dense brute-force K."""
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


def _dense_K(lat, U, kappa, csw):
    """K = M-hat^dag M-hat as a dense matrix on even sites, built from dense blocks of the
    full matrix M = A - kappa H (brute force, independent of the even-odd code path)."""
    from oracle.dirac import WilsonClover, dense

    W = WilsonClover(lat, U, kappa, csw)
    M_ee = dense(lat, W.block(W.M, 0, 0), 0)
    full = dense_full(lat, W.M)
    e = (lat.parity == 0).reshape(-1)
    o = ~e
    idx_e = torch.nonzero(e.repeat_interleave(12)).reshape(-1)
    idx_o = torch.nonzero(o.repeat_interleave(12)).reshape(-1)
    Mee = full[idx_e][:, idx_e]
    Meo = full[idx_e][:, idx_o]
    Moe = full[idx_o][:, idx_e]
    Moo = full[idx_o][:, idx_o]
    assert torch.allclose(Mee, M_ee)
    Mhat = Mee - Meo @ torch.linalg.solve(Moo, Moe)
    return Mhat.conj().T @ Mhat


def dense_full(lat, op):
    """op on the whole lattice as a dense (12 V) x (12 V) matrix, canonical site order."""
    n = lat.V * 12
    e = torch.eye(n, dtype=C128).reshape(n, *lat.shape, 4, 3)
    return op(e).reshape(n, n).T.contiguous()


def test_residual_loss_against_dense_operator():
    """residual_loss = ||K N(b) - b||^2 / ||b||^2 with K assembled densely from the blocks
    of the full Wilson-clover matrix (2^4, every column by brute force)."""
    from oracle.dirac import WilsonClover, to_parity_vector

    lat, U, b = _setup((2, 2, 2, 2), 4)
    kappa, csw = 0.13, 1.0
    ws = nn.init_weights([1, 2, 1], 8)
    Kd = _dense_K(lat, U, kappa, csw)
    y = to_parity_vector(lat, nn.network_apply(lat, U, ws, b))
    bv = to_parity_vector(lat, b)
    want = (torch.linalg.vector_norm(Kd @ y - bv) ** 2 / torch.linalg.vector_norm(bv) ** 2).item()
    W = WilsonClover(lat, U, kappa, csw)
    got = nn.residual_loss(lat, U, ws, b, W.K).item()
    assert abs(got - want) < 1e-12 * max(1.0, want), (got, want)
    assert got > 1e-3   # a non-trivial value: the initial network is far from K^{-1}


def test_residual_gradient_against_finite_differences():
    """dL/dRe W + i dL/dIm W of the residual loss by autograd against central differences
    of residual_loss (4x2x2x4, two layers, random entries of both layers)."""
    from oracle.dirac import WilsonClover

    lat, U, b = _setup((4, 2, 2, 4), 12)
    W = WilsonClover(lat, U, 0.125, 1.0)
    ws = nn.init_weights([1, 2, 1], 9)
    L, gr = nn.residual_grads(lat, U, ws, b, W.K)
    assert abs(L.item() - nn.residual_loss(lat, U, ws, b, W.K).item()) < 1e-14
    rng = np.random.default_rng(1)
    for trial in range(6):
        l = trial % 2
        idx = tuple(int(rng.integers(0, n)) for n in ws[l].shape)
        for part in (1.0, 1j):
            d = 1e-6
            wp = [w.clone() for w in ws]
            wm = [w.clone() for w in ws]
            wp[l][idx] += d * part
            wm[l][idx] -= d * part
            fd = (nn.residual_loss(lat, U, wp, b, W.K) - nn.residual_loss(lat, U, wm, b, W.K)).item() / (2 * d)
            an = gr[l][idx].real.item() if part == 1.0 else gr[l][idx].imag.item()
            assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (trial, part, fd, an)
