"""Action terms, heatbath and forces of PF-MP HMC (oracle, test infrastructure).

PF-MP action (Sec. 2.5, eq. pfmp_action), with the gauge and clover-determinant parts:
  S = S_G + S_det + phi_1^dag P(J) phi_1 + phi_2^dag [J P(J)]^{-1} phi_2 + S_3,
  S_G   = beta sum_{x, mu<nu} (1 - Re tr U_{mu nu}(x) / 3)             (Wilson, Table 3.1)
  S_det = -2 sum_{x odd} log det A(x)      (even-odd clover: det M = det A_oo det M-hat)
  S_3   = phi_3^dag W K^{-1} W^dag phi_3    (the paper's "J K^{-1}" term)
K = M-hat^dag M-hat at kappa, J = W^dag W with W = M-hat at kappa' (same c_sw).

Reading of S_3: the paper writes phi^dag J K^{-1} phi and its force (App. C, eq.
force_hasencorr) as if J, K, W and M-hat all commute (true only for free fields).  The
Hermitian operator W K^{-1} W^dag = W (K^{-1} J) W^{-1} is similar to K^{-1} J, has the
required determinant det J / det K, and reduces to the identity when kappa' = kappa.
Its force is
  dS_3 = 2 Re[chi^dag (dW^dag) phi] - chi^dag dK chi,   chi = K^{-1} W^dag phi,
whose second term has the paper's form with W^dag in place of W.

Forces: F = sum_a T_a dS/d omega_a for U -> exp(i omega_a T_a) U (so that H = sum tr P^2
+ S is conserved by the steps of Sec. 2.1).  They are returned as the coefficients
f[..., mu, a] = dS/d omega_a.  Fermion forces follow App. C: the vectors eta_i, chi_i
(eq. force_poly), eta-bar_i, chi-bar_i (eq. force_polycorr) and chi (eq.
force_hasencorr) are built first; the contraction eta^dag (dK/dU) chi is then taken by
automatic differentiation of the bilinear form with the vectors held fixed.
"""
import math
from dataclasses import dataclass

import torch

from . import cheby
from .dirac import WilsonClover
from .lattice import C128, F64, Lattice, su3_generators
from .solvers import cg, multishift_cg


@dataclass
class PFMPParams:
    beta: float = 5.5
    kappa: float = 0.120
    kappa_h: float = 0.110
    csw: float = 1.0
    n: int = 8
    mu: float = 1.2
    nu: float = 0.9
    tol: float = 1e-12


def _vdot(a, b):
    return (a.conj() * b).sum()


def plaquette_field(lat, U, mu, nu):
    Um, Un = U[..., mu, :, :], U[..., nu, :, :]
    d = lambda X: X.conj().transpose(-1, -2)
    return Um @ lat.fwd(Un, mu) @ d(lat.fwd(Um, nu)) @ d(Un)


def gauge_action(lat, U, beta):
    s = torch.zeros((), dtype=F64)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = plaquette_field(lat, U, mu, nu)
            s = s + (1.0 - torch.diagonal(P, dim1=-2, dim2=-1).sum(-1).real / 3.0).sum()
    return beta * s


def mean_plaquette(lat, U):
    s = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = plaquette_field(lat, U, mu, nu)
            s += torch.diagonal(P, dim1=-2, dim2=-1).sum(-1).real.mean().item() / 3.0
    return s / 6.0


def det_action(lat, U, kappa, csw):
    return -2.0 * WilsonClover(lat, U, kappa, csw).logdet_oo()


def deriv(lat: Lattice, U, fn):
    """f[..., mu, a] = d fn(exp(i omega.T) U) / d omega_a at omega = 0.

    exp(i X) = 1 + i X + O(X^2), so the first derivative is that of fn((1 + i X) U)."""
    T = su3_generators()
    omega = torch.zeros(*lat.shape, 4, 8, dtype=F64, requires_grad=True)
    X = torch.einsum("...a,aij->...ij", omega.to(C128), T)
    Uw = (torch.eye(3, dtype=C128) + 1j * X) @ U
    val = fn(Uw)
    (g,) = torch.autograd.grad(val, omega)
    return g.detach()


class PFMP:
    """The PF-MP action at fixed parameters; fields are full-lattice, even-site tensors."""

    def __init__(self, lat: Lattice, p: PFMPParams):
        self.lat, self.p = lat, p
        self.shifts, self.r = cheby.residues(p.n, p.mu, p.nu)
        self.a_n = cheby.norm(p.n, p.mu, p.nu)
        self.z = cheby.roots(p.n, p.mu, p.nu)

    def ops(self, U):
        M = WilsonClover(self.lat, U, self.p.kappa, self.p.csw)
        W = WilsonClover(self.lat, U, self.p.kappa_h, self.p.csw)
        return M, W

    # ---------------------------------------------------------------- heatbath
    def heatbath(self, U, xi1, xi2, xi3):
        """phi_1 = R(J)^{-1} xi_1, phi_2 = R(J)^dag W^dag xi_2, phi_3 = W J^{-1} M^dag xi_3
        (= W^{-dag} M^dag xi_3), so that each S_i(phi_i) = xi_i^dag xi_i."""
        p = self.p
        M, W = self.ops(U)
        J = W.K
        zh, sh = cheby.half_residues(p.n, p.mu, p.nu)
        xs, _ = multishift_cg(J, xi1, -zh, tol=p.tol)
        phi1 = (sh.reshape(-1, *([1] * xi1.dim())) * xs).sum(0) / math.sqrt(self.a_n)
        phi2 = cheby.apply_R(J, W.mhat_dag(xi2), p.n, p.mu, p.nu, dagger=True)
        y, _, _ = cg(J, M.mhat_dag(xi3), tol=p.tol)
        return phi1, phi2, W.mhat(y)

    # ---------------------------------------------------------------- actions
    def S_poly(self, U, phi1):
        _, W = self.ops(U)
        return _vdot(phi1, cheby.apply_poly(W.K, phi1, self.p.n, self.p.mu, self.p.nu)).real

    def S_polycorr(self, U, phi2):
        _, W = self.ops(U)
        xs, _ = multishift_cg(W.K, phi2, -self.shifts, tol=self.p.tol)
        return sum(self.r[i] * _vdot(phi2, xs[i]) for i in range(self.shifts.numel())).real

    def S_hasen(self, U, phi3):
        M, W = self.ops(U)
        w = W.mhat_dag(phi3)
        x, _, _ = cg(M.K, w, tol=self.p.tol)
        return _vdot(w, x).real

    def S_gauge(self, U):
        return gauge_action(self.lat, U, self.p.beta)

    def S_det(self, U):
        return det_action(self.lat, U, self.p.kappa, self.p.csw)

    # ---------------------------------------------------------------- forces
    def F_gauge(self, U):
        return deriv(self.lat, U, lambda V: gauge_action(self.lat, V, self.p.beta))

    def F_det(self, U):
        return deriv(self.lat, U, lambda V: det_action(self.lat, V, self.p.kappa, self.p.csw))

    def _J_at(self, V):
        return WilsonClover(self.lat, V, self.p.kappa_h, self.p.csw)

    def F_poly(self, U, phi1):
        """F_1 = sum_i eta_i^dag (dJ/dU) chi_i (App. C eq. force_poly); 2n - 2 J products."""
        p = self.p
        _, W = self.ops(U)
        J = W.K
        n = p.n
        z = self.z
        chi = [None] * n
        w = self.a_n * phi1
        chi[n - 1] = w
        for i in range(n - 2, -1, -1):          # chi_i = a_n prod_{j>i} (J - z_j) phi
            w = J(w) - z[i + 1] * w
            chi[i] = w
        eta = [None] * n
        w = phi1
        eta[0] = w
        for i in range(1, n):                    # eta_i = prod_{j<i} (J - z_j^*) phi
            w = J(w) - z[i - 1].conj() * w
            eta[i] = w
        E = torch.stack(eta)
        X = torch.stack(chi)
        return deriv(self.lat, U, lambda V: _vdot(E, self._J_at(V).K(X)).real)

    def F_polycorr(self, U, phi2):
        """F_2 = -sum_i eta-bar_i^dag (dJ/dU) chi-bar_i (App. C eq. force_polycorr)."""
        _, W = self.ops(U)
        xs, _ = multishift_cg(W.K, phi2, -self.shifts, tol=self.p.tol)
        # eta-bar_i = (J - z_i^*)^{-1} phi: the solution at the conjugate shift
        conj_index = []
        for i in range(self.shifts.numel()):
            d = (self.shifts - self.shifts[i].conj()).abs()
            conj_index.append(int(torch.argmin(d)))
        E = xs[conj_index]
        X = self.r.reshape(-1, *([1] * phi2.dim())) * xs
        return deriv(self.lat, U, lambda V: -_vdot(E, self._J_at(V).K(X)).real)

    def F_hasen(self, U, phi3):
        """dS_3 = 2 Re[chi^dag (dW^dag) phi] - chi^dag dK chi with chi = K^{-1} W^dag phi."""
        M, W = self.ops(U)
        chi, _, _ = cg(M.K, W.mhat_dag(phi3), tol=self.p.tol)
        kap, kh, csw = self.p.kappa, self.p.kappa_h, self.p.csw

        def f(V):
            Mv = WilsonClover(self.lat, V, kap, csw)
            Wv = WilsonClover(self.lat, V, kh, csw)
            return 2.0 * _vdot(chi, Wv.mhat_dag(phi3)).real - _vdot(chi, Mv.K(chi)).real

        return deriv(self.lat, U, f)
