"""Gauge-covariant network used as a flexible preconditioner (oracle, test infrastructure).

The paper has no learned component; the network is the project's reading of the
preconditioner the method's solves are given:

  layer l (C_in -> C_out channels), for every site x and output channel c:
    y_c(x) = sum_{c'} [ W0_{c c'} x_{c'}(x)
                        + sum_mu ( Wf_mu_{c c'} U_mu(x) x_{c'}(x + mu)
                                 + Wb_mu_{c c'} U_mu(x - mu)^dag x_{c'}(x - mu) ) ]
  with every W a complex 4x4 matrix acting on spin (9 of them per channel pair: the site
  itself, 4 forward and 4 backward hops), U acting on colour, and the fermion boundary
  factor on hops across the time boundary.  No nonlinearity: the network is a fixed
  linear operator, so FGCR sees one preconditioner throughout.

  network: channels 1 -> C -> ... -> C -> 1; the input is an even-site field embedded
  with zeros on odd sites, the output is read on even sites.

Weights are stored as W[layer][d][c_out][c_in][4][4] complex with d = 0 (site),
1 + mu (forward hop), 5 + mu (backward hop).  Gradients are taken by torch.autograd
(complex convention: dL/dRe + i dL/dIm).
"""
import torch

from .lattice import C128, Lattice


def layer_apply(lat: Lattice, U, W, x):
    """One layer.  x: (C_in, Lt, Lz, Ly, Lx, 4, 3) complex; W: (9, C_out, C_in, 4, 4)."""
    def mix(Wd, v):
        return torch.einsum("oiuv,itzyxva->otzyxua", Wd, v)

    def cmul(Um, v):
        return sum(Um[..., None, :, b] * v[..., :, b:b + 1] for b in range(3))

    def cmul_dag(Um, v):
        Uc = Um.conj()
        return sum(Uc[..., None, b, :] * v[..., :, b:b + 1] for b in range(3))

    y = mix(W[0], x)
    for mu in range(4):
        Um = U[..., mu, :, :]
        fw = cmul(Um, lat.ffwd(x, mu))
        y = y + mix(W[1 + mu], fw)
        bw = cmul_dag(lat.bwd(Um, mu), lat.fbwd(x, mu))
        y = y + mix(W[5 + mu], bw)
    return y


def network_apply(lat, U, weights, b_even):
    """weights: list of (9, C_out, C_in, 4, 4) tensors.  b_even: (Lt, Lz, Ly, Lx, 4, 3)."""
    x = (lat.even * b_even).unsqueeze(0)
    for W in weights:
        x = layer_apply(lat, U, W, x)
    return lat.even * x[0]


def loss(lat, U, weights, b, x_true):
    """|| N(b) - x ||^2 / ||x||^2 on even sites."""
    y = network_apply(lat, U, weights, b)
    d = lat.even * (y - x_true)
    return (d.abs() ** 2).sum() / ((lat.even * x_true).abs() ** 2).sum()


def residual_loss(lat, U, weights, b, K):
    """|| K N(b) - b ||^2 / ||b||^2 on even sites: K N close to the identity, the
    property a right preconditioner of K needs (K = M-hat^dag M-hat)."""
    y = network_apply(lat, U, weights, b)
    d = lat.even * (K(y) - b)
    return (d.abs() ** 2).sum() / ((lat.even * b).abs() ** 2).sum()


def residual_grads(lat, U, weights, b, K):
    ws = [w.clone().requires_grad_(True) for w in weights]
    L = residual_loss(lat, U, ws, b, K)
    g = torch.autograd.grad(L, ws)
    return L.detach(), [t.detach() for t in g]


def init_weights(channels, seed):
    """Initial weights drawn by pfmp_inputs (shared with the GPU side)."""
    import pfmp_inputs as pin

    return [torch.tensor(w) for w in pin.nn_weights(channels, seed)]


def grads(lat, U, weights, b, x_true):
    ws = [w.clone().requires_grad_(True) for w in weights]
    L = loss(lat, U, ws, b, x_true)
    g = torch.autograd.grad(L, ws)
    return L.detach(), [t.detach() for t in g]
