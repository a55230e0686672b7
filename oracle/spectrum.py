"""Spectral range of K (oracle, test infrastructure).

App. A: the Chebyshev filter is a good approximation of K^{-1} only inside its ellipse,
which runs from 0 to 2 mu along the real axis, so (mu, nu) must be chosen with the
spectrum [lambda_min, lambda_max] of K inside it (the paper quotes lambda_min = 3.2e-5 and
lambda_max = 2.2 for its configuration and takes mu > lambda_max / 2).

* ``extreme_eigenvalues``: the definition -- all eigenvalues of the dense K assembled
  column by column, smallest and largest (small lattices only).
* ``lanczos``: the Lanczos recurrence (Lanczos 1950) written out plainly, without
  reorthogonalisation: beta_0 = 0, v_1 = s/|s|, alpha_j = <v_j, K v_j>,
  w = K v_j - alpha_j v_j - beta_{j-1} v_{j-1}, beta_j = |w|, v_{j+1} = w / beta_j.
* ``ritz_extremes``: extreme eigenvalues of the tridiagonal T_k by a library eigensolver.
"""
import torch

from .dirac import WilsonClover, dense


def extreme_eigenvalues(lat, U, kappa, csw):
    K = dense(lat, WilsonClover(lat, U, kappa, csw).K)
    ev = torch.linalg.eigvalsh(0.5 * (K + K.conj().T))
    return ev[0].item(), ev[-1].item()


def lanczos(K, v0, k):
    """(alpha[k], beta[k]) of k Lanczos steps on the Hermitian operator K from v0."""
    v_prev = torch.zeros_like(v0)
    v = v0 / torch.sqrt((v0.abs() ** 2).sum())
    alpha, beta = [], []
    b_prev = 0.0
    for _ in range(k):
        Kv = K(v)
        a = (v.conj() * Kv).sum().real.item()
        w = Kv - a * v - b_prev * v_prev
        b = torch.sqrt((w.abs() ** 2).sum()).item()
        alpha.append(a)
        beta.append(b)
        v_prev, v, b_prev = v, w / b, b
    return torch.tensor(alpha, dtype=torch.float64), torch.tensor(beta, dtype=torch.float64)


def ritz_extremes(alpha, beta):
    k = alpha.numel()
    T = torch.diag(alpha) + torch.diag(beta[:k - 1], 1) + torch.diag(beta[:k - 1], -1)
    ev = torch.linalg.eigvalsh(T)
    return ev[0].item(), ev[-1].item()
