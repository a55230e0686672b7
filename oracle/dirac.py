"""Wilson-clover fermion operator, even-odd Schur complement, K and J (oracle).

The paper's operator (Sec. 2.1, Sec. 2.2 eq. hasenbusch, Table 3.1 "even-odd Wilson"):
  K = M-hat^dagger M-hat, with M-hat the even-odd reduced Dirac matrix, and
  J = W^dagger W, W the same matrix at a heavier mass (kappa' < kappa).
The paper uses Wilson fermions only; the clover term is added with the convention

  M    = A - kappa H,
  (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)
  A(x) = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x)
       = 1 - (kappa c_sw / 2) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x),
  F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag) / (8 i), trace removed,
  Q_{mu nu}(x) = sum of the four plaquette leaves at x in the (mu, nu) plane.

Even-odd: with P_e, P_o the parity projectors, M-hat = M_ee - M_eo M_oo^{-1} M_oe, built
from the blocks of the full matrix (M_oo is site-diagonal, inverted site by site).  Then
det M = det M_oo det M-hat.

Spinor fields are complex tensors (..., Lt, Lz, Ly, Lx, 4, 3); an "even field" is a
full-lattice field that is zero on odd sites.
"""
import torch

from .lattice import C128, Lattice, dagger, gammas, sigma_munu

_G, _G5 = gammas()
_I4 = torch.eye(4, dtype=C128)


def _cmul(U, psi):
    """Colour matrix field times spinor field: (U psi)_{s,a} = sum_b U_{ab} psi_{s,b}."""
    return sum(U[..., None, :, b] * psi[..., :, b:b + 1] for b in range(3))


def _cmul_dag(U, psi):
    """(U^dag psi)_{s,a} = sum_b conj(U_{ba}) psi_{s,b}."""
    Uc = U.conj()
    return sum(Uc[..., None, b, :] * psi[..., :, b:b + 1] for b in range(3))


def _smul(S, psi):
    """4x4 spin matrix times spinor field."""
    return torch.einsum("rs,...sa->...ra", S, psi)


def gamma5(psi):
    return _smul(_G5, psi)


def clover_leaves(lat: Lattice, U, mu, nu):
    """Q_{mu nu}(x): the four plaquettes in the (mu, nu) plane that start and end at x,
    all traversed in the same (mu then nu) orientation."""
    Um, Un = U[..., mu, :, :], U[..., nu, :, :]
    f, b = lat.fwd, lat.bwd
    Un_xpm = f(Un, mu)                   # U_nu(x+mu)
    Um_xpn = f(Um, nu)                   # U_mu(x+nu)
    Um_xmm = b(Um, mu)                   # U_mu(x-mu)
    Un_xmm = b(Un, mu)                   # U_nu(x-mu)
    Um_xmmpn = f(Um_xmm, nu)             # U_mu(x-mu+nu)
    Um_xmmmn = b(Um_xmm, nu)             # U_mu(x-mu-nu)
    Un_xmmmn = b(Un_xmm, nu)             # U_nu(x-mu-nu)
    Un_xmn = b(Un, nu)                   # U_nu(x-nu)
    Um_xmn = b(Um, nu)                   # U_mu(x-nu)
    Un_xpmmn = b(Un_xpm, nu)             # U_nu(x+mu-nu)
    d = dagger
    L1 = Um @ Un_xpm @ d(Um_xpn) @ d(Un)
    L2 = Un @ d(Um_xmmpn) @ d(Un_xmm) @ Um_xmm
    L3 = d(Um_xmm) @ d(Un_xmmmn) @ Um_xmmmn @ Un_xmn
    L4 = d(Un_xmn) @ Um_xmn @ Un_xpmmn @ d(Um)
    return L1 + L2 + L3 + L4


def field_strength(lat, U, mu, nu):
    """F_{mu nu} = (Q - Q^dag)/(8i) with its colour trace removed (Hermitian, traceless)."""
    Q = clover_leaves(lat, U, mu, nu)
    F = (Q - dagger(Q)) / 8j
    tr = torch.diagonal(F, dim1=-2, dim2=-1).sum(-1)
    eye = torch.eye(3, dtype=C128)
    return F - (tr / 3)[..., None, None] * eye


def clover_matrix(lat, U, kappa, csw):
    """A(x) as a 12x12 matrix per site, index = 3*spin + colour."""
    A = torch.zeros(*lat.shape, 12, 12, dtype=C128)
    A = A + torch.eye(12, dtype=C128)
    if csw == 0.0:
        return A
    for mu in range(4):
        for nu in range(mu + 1, 4):
            F = field_strength(lat, U, mu, nu)
            s = sigma_munu(_G, mu, nu)
            A = A - kappa * csw * torch.einsum("rs,...ab->...rasb", s, F).reshape(*lat.shape, 12, 12)
    return A


def apply_site_matrix(A, psi):
    """Per-site 12x12 matrix on a spinor field (..., Lt, Lz, Ly, Lx, 4, 3)."""
    sh = psi.shape
    v = psi.reshape(*sh[:-2], 12)
    return torch.einsum("tzyxij,...tzyxj->...tzyxi", A, v).reshape(sh)


def hop(lat: Lattice, U, psi, adjoint=False):
    """Wilson hop H psi (or H^dagger psi, which swaps the projector signs)."""
    s = -1.0 if adjoint else 1.0
    out = torch.zeros_like(psi)
    for mu in range(4):
        Um = U[..., mu, :, :]
        fw = _cmul(Um, lat.ffwd(psi, mu))
        out = out + fw - s * _smul(_G[mu], fw)
        bw = _cmul_dag(lat.bwd(Um, mu), lat.fbwd(psi, mu))
        out = out + bw + s * _smul(_G[mu], bw)
    return out


class WilsonClover:
    """Full-lattice Wilson-clover matrix M = A - kappa H at one (kappa, c_sw)."""

    def __init__(self, lat: Lattice, U, kappa, csw):
        self.lat, self.U, self.kappa, self.csw = lat, U, kappa, csw
        self.A = clover_matrix(lat, U, kappa, csw)
        self._Ainv = None

    @property
    def Ainv(self):
        if self._Ainv is None:
            self._Ainv = torch.linalg.inv(self.A)
        return self._Ainv

    def M(self, psi):
        return apply_site_matrix(self.A, psi) - self.kappa * hop(self.lat, self.U, psi)

    def Mdag(self, psi):
        # A is Hermitian site by site, so M^dag = A - kappa H^dag
        return apply_site_matrix(self.A, psi) - self.kappa * hop(self.lat, self.U, psi, adjoint=True)

    # --- blocks of the full matrix ----------------------------------------------------
    def block(self, op, p, q):
        mp, mq = self.lat.mask(p), self.lat.mask(q)
        return lambda psi: mp * op(mq * psi)

    def diag_inv(self, p):
        """(M_pp)^{-1}: M_pp is site-diagonal (the clover A), inverted site by site."""
        mp = self.lat.mask(p)
        return lambda psi: mp * apply_site_matrix(self.Ainv, mp * psi)

    def mhat(self, psi_e):
        """M-hat psi_e = M_ee psi - M_eo M_oo^{-1} M_oe psi (psi even)."""
        Mee, Meo, Moe = self.block(self.M, 0, 0), self.block(self.M, 0, 1), self.block(self.M, 1, 0)
        return Mee(psi_e) - Meo(self.diag_inv(1)(Moe(psi_e)))

    def mhat_dag(self, psi_e):
        """The adjoint of M-hat: the same Schur complement of M^dagger."""
        D = self.Mdag
        Mee, Meo, Moe = self.block(D, 0, 0), self.block(D, 0, 1), self.block(D, 1, 0)
        return Mee(psi_e) - Meo(self.diag_inv(1)(Moe(psi_e)))

    def K(self, psi_e):
        return self.mhat_dag(self.mhat(psi_e))

    def logdet_oo(self):
        """sum over odd sites of log det A(x) (A Hermitian positive for small fields)."""
        sign, la = torch.linalg.slogdet(self.A)
        return (la * (self.lat.parity == 1)).sum()


def dense(lat: Lattice, op, parity=0, chunk=512):
    """Assemble op restricted to one parity as a dense complex matrix (brute force)."""
    mask = (lat.parity == parity).reshape(-1)
    sites = torch.nonzero(mask).reshape(-1)
    n = sites.numel() * 12
    cols = []
    for start in range(0, n, chunk):
        idx = torch.arange(start, min(n, start + chunk))
        e = torch.zeros(idx.numel(), lat.V * 12, dtype=C128)
        e[torch.arange(idx.numel()), sites[idx // 12] * 12 + idx % 12] = 1
        e = e.reshape(idx.numel(), *lat.shape, 4, 3)
        y = op(e).reshape(idx.numel(), lat.V, 12)[:, sites, :].reshape(idx.numel(), n)
        cols.append(y)
    return torch.cat(cols, 0).T.contiguous()


def to_parity_vector(lat, psi, parity=0):
    """Even (or odd) sites of a full field, in canonical site order, flattened."""
    mask = (lat.parity == parity).reshape(-1)
    return psi.reshape(*psi.shape[:-6], lat.V, 12)[..., mask, :].reshape(*psi.shape[:-6], -1)


def from_parity_vector(lat, v, parity=0):
    mask = (lat.parity == parity).reshape(-1)
    out = torch.zeros(*v.shape[:-1], lat.V, 12, dtype=C128)
    out[..., mask, :] = v.reshape(*v.shape[:-1], -1, 12)
    return out.reshape(*v.shape[:-1], *lat.shape, 4, 3)
