"""Chebyshev polynomial filter P_n(z) ~ 1/z (App. A) and its partial fractions (App. C).

  P_n(z)  = a_n prod_{k=1}^{n} (z - z_k)
  z_k     = mu (1 - cos theta_k) - i sqrt(mu^2 - nu^2) sin theta_k,  theta_k = 2 pi k / (n+1)
  a_n     = 1 / (mu prod_k (mu - z_k))

Correction term [z P_n(z)]^{-1} (App. C, eq. force_polycorr): with z_{n+1} = 0,
  1 / (z P_n(z)) = sum_{i=1}^{n+1} r_i / (z - z_i),
  r_i = (1 / a_n) prod_{j != i, j <= n+1} 1 / (z_i - z_j)     (the residue at z_i).
Two readings of the printed formula: (1) it omits the 1/a_n factor that [P K]^{-1}
carries (the force expression drops c_n); it is restored so that the sum equals
[z P(z)]^{-1}; (2) it writes 1/(z_j - z_i), which differs from the residue by
(-1)^(number of poles - 1) -- the same for the n+1 poles of an even order n, which is
the only case used, but wrong for an even number of poles (the half products below).

Heatbath split (derived; the paper calls the heatbath negligible and gives no form):
for even n the roots come in conjugate pairs and a_n > 0, so
  R(z) = sqrt(a_n) prod_{k: Im z_k < 0} (z - z_k),  P_n(z) = conj(R)(z) R(z) on the real axis,
i.e. P(J) = R(J)^dag R(J) for Hermitian J.

Factorised filters (App. A, Sec. 2.3 eq. 2poly): with (p1 + 1) | (p2 + 1) the ratio
Q = P_p2 / P_p1 is the polynomial whose roots are those of P_p2 that P_p1 does not have,
normalised by a_p2 / a_p1 (``filter_roots``); it splits as R_Q^dag R_Q the same way.
"""
import math

import torch


def roots(n, mu, nu):
    k = torch.arange(1, n + 1, dtype=torch.float64)
    th = 2 * math.pi * k / (n + 1)
    re = mu * (1 - torch.cos(th))
    im = -math.sqrt(mu * mu - nu * nu) * torch.sin(th)
    return torch.complex(re, im)


def norm(n, mu, nu):
    z = roots(n, mu, nu)
    return (1.0 / (mu * torch.prod(mu - z))).real.item()


def poly_scalar(x, n, mu, nu):
    """P_n evaluated at (complex) scalar points x."""
    z = roots(n, mu, nu)
    x = torch.as_tensor(x, dtype=torch.complex128)
    return norm(n, mu, nu) * torch.prod(x[..., None] - z, dim=-1)


def residues(n, mu, nu):
    """(shifts, r): shifts z_1..z_n, z_{n+1} = 0 and the residues r_i of 1/(z P_n(z))."""
    z = torch.cat([roots(n, mu, nu), torch.zeros(1, dtype=torch.complex128)])
    a = norm(n, mu, nu)
    r = []
    for i in range(n + 1):
        others = torch.cat([z[:i], z[i + 1:]])
        r.append(1.0 / (a * torch.prod(z[i] - others)))
    return z, torch.stack(r)


def half_roots(n, mu, nu):
    """Roots with negative imaginary part (the factor R of P = R^dag R)."""
    if n % 2:
        raise ValueError("odd polynomial orders are not supported (a real root at 2 mu)")
    z = roots(n, mu, nu)
    return z[z.imag < 0]


def half_residues(n, mu, nu):
    """Residues of 1/prod_{Im z_k<0}(z - z_k) = sum_k s_k / (z - z_k) over the half set."""
    z = half_roots(n, mu, nu)
    s = []
    for i in range(z.numel()):
        others = torch.cat([z[:i], z[i + 1:]])
        s.append(1.0 / torch.prod(z[i] - others))
    return z, torch.stack(s)


def apply_poly(J, v, n, mu, nu):
    """P_n(J) v = a_n prod_{k=1}^{n} (J - z_k) v, factors applied in the order k = 1..n."""
    z = roots(n, mu, nu)
    w = v
    for k in range(n):
        w = J(w) - z[k] * w
    return norm(n, mu, nu) * w


def apply_R(J, v, n, mu, nu, dagger=False):
    """R(J) v or R(J)^dag v (conjugated roots), R = sqrt(a_n) prod_{Im z<0} (J - z)."""
    z = half_roots(n, mu, nu)
    if dagger:
        z = z.conj()
    w = v
    for k in range(z.numel()):
        w = J(w) - z[k] * w
    return math.sqrt(norm(n, mu, nu)) * w


def filter_roots(p1, p2, mu, nu):
    """Roots q_k and normalisation c of the filter Q(z) = P_p2(z) / P_p1(z) = c prod_k (z - q_k).

    App. A: two approximations with the same (mu, nu) factorise when (p1 + 1) divides
    (p2 + 1); the roots of P_p1 (angles 2 pi j / (p1 + 1)) are then the roots of P_p2 with
    index k = j (p2 + 1) / (p1 + 1), so Q keeps the other p2 - p1 roots of P_p2 and
    c = a_p2 / a_p1.  p1 = 0 gives P_p2 itself (Q = P_p2, c = a_p2)."""
    if p2 < 2 or p2 % 2 or p1 < 0 or p1 % 2:
        raise ValueError("filter orders must be even (p1 >= 0, p2 >= 2)")
    z = roots(p2, mu, nu)
    if p1 == 0:
        return z, norm(p2, mu, nu)
    if p2 <= p1 or (p2 + 1) % (p1 + 1):
        raise ValueError("P_p1 divides P_p2 only when (p1 + 1) divides (p2 + 1)")
    m = (p2 + 1) // (p1 + 1)
    keep = [k - 1 for k in range(1, p2 + 1) if k % m]
    return z[keep], norm(p2, mu, nu) / norm(p1, mu, nu)


def product_half(z):
    """Half set of a conjugate-closed root list (Im < 0) and the residues s_k of
    1 / prod_k (z - zh_k); the heatbath factor of c prod (z - z_k) is sqrt(c) prod (z - zh_k)."""
    zh = z[z.imag < 0]
    s = []
    for i in range(zh.numel()):
        others = torch.cat([zh[:i], zh[i + 1:]])
        s.append(1.0 / torch.prod(zh[i] - others))
    return zh, torch.stack(s)


def apply_product(J, v, z, c):
    """c prod_k (J - z_k) v, factors applied in list order."""
    w = v
    for k in range(z.numel()):
        w = J(w) - z[k] * w
    return c * w
