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


# ====================================================================================
# General filtered / mass-preconditioned actions (Sec. 2.2 eq. hasenbusch, Sec. 2.3 eqs.
# 1poly and 2poly, Sec. 2.5 eq. pfmp_action, Sec. 3.6 (2PF-1MP and 1PF-2MP))
# ====================================================================================
#
# A term list over a list of hopping parameters kappas[0..] (kappas[0] = the target
# operator K; J_a = W_a^dag W_a with W_a = M-hat at kappas[a]; J_0 = K):
#   gauge       S_G
#   det         -2 sum_{x odd} log det A(x) at kappas[a]
#   filter      phi^dag Q(J_a) phi,  Q = P_p2 / P_p1 (p1 = 0: P_p2)
#   filtercorr  phi^dag [J_a P_p2(J_a)]^{-1} phi
#   ratio       phi^dag W_a K_b^{-1} W_a^dag phi   (the paper's "J_a K_b^{-1}", see S_3 above)
#   inv         phi^dag J_a^{-1} phi               (the first mass-preconditioning term)
# Heatbath (derived so that every S_i(phi_i) = xi_i^dag xi_i):
#   filter      phi = R_Q(J_a)^{-1} xi,  R_Q = sqrt(c) prod_{Im q_k < 0} (J_a - q_k)
#   filtercorr  phi = R_p2(J_a)^dag W_a^dag xi
#   ratio       phi = W_a J_a^{-1} M_b^dag xi  (M_b = M-hat at kappas[b])
#   inv         phi = W_a^dag xi
# Forces:
#   filter      App. C eq. force_poly with the roots q_k and c in place of z_k and a_n
#   filtercorr  App. C eq. force_polycorr at order p2
#   ratio       2 Re chi^dag (dW_a^dag) phi - chi^dag dK_b chi,  chi = K_b^{-1} W_a^dag phi
#   inv         -chi^dag dJ_a chi,  chi = J_a^{-1} phi

FERMION_KINDS = ("filter", "filtercorr", "ratio", "inv")


@dataclass
class Term:
    kind: str
    a: int = 0
    b: int = 0
    p1: int = 0
    p2: int = 0


def scheme(name, p1=0, p2=0):
    """Term lists of the actions the paper compares (Sec. 2, Sec. 3).  Hasenbusch kappas
    are indexed from 1 upwards, lightest-first towards the target kappas[0]:
      1PF      Sec. 2.3 eq. 1poly on K:            P_p2(K), [K P_p2(K)]^{-1}
      2PF      Sec. 2.3 eq. 2poly on K:            P_p1(K), Q(K), [K P_p2(K)]^{-1}
      1MP      Sec. 2.2 eq. hasenbusch:            J_1^{-1}, J_1 K^{-1}
      2MP      two Hasenbusch masses:              J_1^{-1}, J_1 J_2^{-1}, J_2 K^{-1}
      PF-MP    Sec. 2.5 eq. pfmp_action (1PF-1MP): P_p2(J_1), [J_1 P_p2(J_1)]^{-1}, J_1 K^{-1}
      2PF-1MP  Sec. 3.6:  P_p1(J_1), Q(J_1), [J_1 P_p2(J_1)]^{-1}, J_1 K^{-1}
      1PF-2MP  Sec. 3.6:  P_p2(J_1), [J_1 P_p2(J_1)]^{-1}, J_1 J_2^{-1}, J_2 K^{-1}
    Every list starts with the gauge and clover-determinant terms."""
    base = [Term("gauge"), Term("det", a=0)]
    f = {
        "1PF": [Term("filter", a=0, p2=p2), Term("filtercorr", a=0, p2=p2)],
        "2PF": [Term("filter", a=0, p2=p1), Term("filter", a=0, p1=p1, p2=p2), Term("filtercorr", a=0, p2=p2)],
        "1MP": [Term("inv", a=1), Term("ratio", a=1, b=0)],
        "2MP": [Term("inv", a=1), Term("ratio", a=1, b=2), Term("ratio", a=2, b=0)],
        "PF-MP": [Term("filter", a=1, p2=p2), Term("filtercorr", a=1, p2=p2), Term("ratio", a=1, b=0)],
        "2PF-1MP": [Term("filter", a=1, p2=p1), Term("filter", a=1, p1=p1, p2=p2), Term("filtercorr", a=1, p2=p2),
                    Term("ratio", a=1, b=0)],
        "1PF-2MP": [Term("filter", a=1, p2=p2), Term("filtercorr", a=1, p2=p2), Term("ratio", a=1, b=2),
                    Term("ratio", a=2, b=0)],
    }[name]
    return base + f


class Action:
    """A general action: ``terms`` over the hopping parameters ``kappas`` (same c_sw).
    Pseudofermions belong to the fermion terms in list order."""

    def __init__(self, lat: Lattice, beta, csw, kappas, terms, mu=1.2, nu=0.9, tol=1e-12):
        self.lat, self.beta, self.csw = lat, beta, csw
        self.kappas, self.terms = list(kappas), list(terms)
        self.mu, self.nu, self.tol = mu, nu, tol
        for t in self.terms:
            if t.kind == "filter":
                cheby.filter_roots(t.p1, t.p2, mu, nu)       # validates the orders
            if t.kind == "filtercorr" and (t.p2 < 2 or t.p2 % 2):
                raise ValueError("filter orders must be even")
        self.pf = [i for i, t in enumerate(self.terms) if t.kind in FERMION_KINDS]

    def op(self, U, a):
        return WilsonClover(self.lat, U, self.kappas[a], self.csw)

    # ---------------------------------------------------------------- heatbath
    def heatbath(self, U, xis):
        """One pseudofermion per fermion term, from the noise xis (same order)."""
        phis = []
        for i, xi in zip(self.pf, xis):
            t = self.terms[i]
            W = self.op(U, t.a)
            if t.kind == "filter":
                z, c = cheby.filter_roots(t.p1, t.p2, self.mu, self.nu)
                zh, s = cheby.product_half(z)
                xs, _ = multishift_cg(W.K, xi, -zh, tol=self.tol)
                phis.append((s.reshape(-1, *([1] * xi.dim())) * xs).sum(0) / math.sqrt(c))
            elif t.kind == "filtercorr":
                phis.append(cheby.apply_R(W.K, W.mhat_dag(xi), t.p2, self.mu, self.nu, dagger=True))
            elif t.kind == "ratio":
                Mb = self.op(U, t.b)
                y, _, _ = cg(W.K, Mb.mhat_dag(xi), tol=self.tol)
                phis.append(W.mhat(y))
            else:  # inv
                phis.append(W.mhat_dag(xi))
        return phis

    # ---------------------------------------------------------------- actions
    def S(self, U, i, phi=None):
        t = self.terms[i]
        if t.kind == "gauge":
            return gauge_action(self.lat, U, self.beta)
        if t.kind == "det":
            return det_action(self.lat, U, self.kappas[t.a], self.csw) if self.csw != 0 else torch.zeros((), dtype=F64)
        W = self.op(U, t.a)
        if t.kind == "filter":
            z, c = cheby.filter_roots(t.p1, t.p2, self.mu, self.nu)
            return _vdot(phi, cheby.apply_product(W.K, phi, z, c)).real
        if t.kind == "filtercorr":
            shifts, r = cheby.residues(t.p2, self.mu, self.nu)
            xs, _ = multishift_cg(W.K, phi, -shifts, tol=self.tol)
            return sum(r[k] * _vdot(phi, xs[k]) for k in range(shifts.numel())).real
        if t.kind == "ratio":
            w = W.mhat_dag(phi)
            x, _, _ = cg(self.op(U, t.b).K, w, tol=self.tol)
            return _vdot(w, x).real
        x, _, _ = cg(W.K, phi, tol=self.tol)            # inv
        return _vdot(phi, x).real

    # ---------------------------------------------------------------- forces
    def F(self, U, i, phi=None):
        t = self.terms[i]
        lat, csw = self.lat, self.csw
        ka = self.kappas[t.a]
        Ja = lambda V: WilsonClover(lat, V, ka, csw).K
        if t.kind == "gauge":
            return deriv(lat, U, lambda V: gauge_action(lat, V, self.beta))
        if t.kind == "det":
            if csw == 0:
                return torch.zeros(*lat.shape, 4, 8, dtype=F64)
            return deriv(lat, U, lambda V: det_action(lat, V, ka, csw))
        W = self.op(U, t.a)
        J = W.K
        if t.kind == "filter":
            z, c = cheby.filter_roots(t.p1, t.p2, self.mu, self.nu)
            m = z.numel()
            chi = [None] * m
            w = c * phi
            chi[m - 1] = w
            for k in range(m - 2, -1, -1):      # chi_k = c prod_{j>k} (J - q_j) phi
                w = J(w) - z[k + 1] * w
                chi[k] = w
            eta = [phi]
            for k in range(1, m):                # eta_k = prod_{j<k} (J - q_j^*) phi
                eta.append(J(eta[-1]) - z[k - 1].conj() * eta[-1])
            E, X = torch.stack(eta), torch.stack(chi)
            return deriv(lat, U, lambda V: _vdot(E, Ja(V)(X)).real)
        if t.kind == "filtercorr":
            shifts, r = cheby.residues(t.p2, self.mu, self.nu)
            xs, _ = multishift_cg(J, phi, -shifts, tol=self.tol)
            conj_index = [int(torch.argmin((shifts - shifts[k].conj()).abs())) for k in range(shifts.numel())]
            E = xs[conj_index]
            X = r.reshape(-1, *([1] * phi.dim())) * xs
            return deriv(lat, U, lambda V: -_vdot(E, Ja(V)(X)).real)
        if t.kind == "ratio":
            kb = self.kappas[t.b]
            chi, _, _ = cg(self.op(U, t.b).K, W.mhat_dag(phi), tol=self.tol)

            def f(V):
                Wv = WilsonClover(lat, V, ka, csw)
                Mv = WilsonClover(lat, V, kb, csw)
                return 2.0 * _vdot(chi, Wv.mhat_dag(phi)).real - _vdot(chi, Mv.K(chi)).real

            return deriv(lat, U, f)
        chi, _, _ = cg(J, phi, tol=self.tol)             # inv
        return deriv(lat, U, lambda V: -_vdot(chi, Ja(V)(chi)).real)
