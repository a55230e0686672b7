"""Lattice geometry, gamma matrices and SU(3) helpers for the oracle (test infrastructure).

Conventions (the paper is silent on all of them):
  * site fields are tensors shaped (..., Lt, Lz, Ly, Lx, <2 internal dims>), i.e. the
    canonical lexicographic order with x fastest; the four site axes sit at -6..-3;
  * direction mu = 0, 1, 2, 3 is x, y, z, t;
  * gauge links are periodic; fermions take a factor ``bc_t`` (-1: antiperiodic) when a
    hop crosses the time boundary;
  * chiral (DeGrand-Rossi) gamma basis with gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 =
    diag(1, 1, -1, -1);
  * su(3) generators T_a = lambda_a / 2 (Gell-Mann), tr T_a T_b = delta_ab / 2.
"""
import math

import torch

C128 = torch.complex128
F64 = torch.float64


def gammas():
    """The four Euclidean gamma matrices (DeGrand-Rossi chiral basis) and gamma_5."""
    i = 1j
    g = [
        [[0, 0, 0, i], [0, 0, i, 0], [0, -i, 0, 0], [-i, 0, 0, 0]],
        [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
        [[0, 0, i, 0], [0, 0, 0, -i], [-i, 0, 0, 0], [0, i, 0, 0]],
        [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
    ]
    G = [torch.tensor(m, dtype=C128) for m in g]
    g5 = G[0] @ G[1] @ G[2] @ G[3]
    return G, g5


def sigma_munu(G, mu, nu):
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]."""
    return 0.5j * (G[mu] @ G[nu] - G[nu] @ G[mu])


def su3_generators():
    """T_a = lambda_a / 2, a = 1..8, as a (8, 3, 3) complex tensor."""
    lam = torch.zeros(8, 3, 3, dtype=C128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1] = -1j
    lam[1, 1, 0] = 1j
    lam[2, 0, 0] = 1
    lam[2, 1, 1] = -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2] = -1j
    lam[4, 2, 0] = 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2] = -1j
    lam[6, 2, 1] = 1j
    s3 = 1.0 / math.sqrt(3.0)
    lam[7, 0, 0] = s3
    lam[7, 1, 1] = s3
    lam[7, 2, 2] = -2 * s3
    return lam / 2


def algebra_to_matrix(h):
    """H = sum_a h_a T_a for real coefficients h[..., 8] -> Hermitian traceless (..., 3, 3)."""
    T = su3_generators()
    return torch.einsum("...a,aij->...ij", h.to(C128), T)


def matrix_to_algebra(X):
    """Coefficients x_a = 2 Re tr(T_a X) of a Hermitian traceless X (inverse of the above)."""
    T = su3_generators()
    return 2.0 * torch.einsum("aij,...ji->...a", T, X).real


def expi_hermitian(H, eps):
    """exp(i eps H) for Hermitian H, by eigendecomposition H = V diag(w) V^dagger."""
    w, V = torch.linalg.eigh(H)
    ph = torch.exp(1j * eps * w.to(C128))
    return (V * ph.unsqueeze(-2)) @ V.conj().transpose(-1, -2)


def dagger(X):
    return X.conj().transpose(-1, -2)


class Lattice:
    """A 4-D periodic box of extent dims = (Lx, Ly, Lz, Lt)."""

    def __init__(self, dims, bc_t=-1):
        self.dims = tuple(int(d) for d in dims)
        Lx, Ly, Lz, Lt = self.dims
        self.shape = (Lt, Lz, Ly, Lx)
        self.V = Lx * Ly * Lz * Lt
        self.bc_t = bc_t
        t, z, y, x = torch.meshgrid(
            torch.arange(Lt), torch.arange(Lz), torch.arange(Ly), torch.arange(Lx), indexing="ij"
        )
        self.coords = (x, y, z, t)
        self.parity = (x + y + z + t) % 2
        # masks broadcastable against (..., Lt, Lz, Ly, Lx, a, b)
        self.even = (self.parity == 0).to(F64)[..., None, None]
        self.odd = (self.parity == 1).to(F64)[..., None, None]

    @staticmethod
    def axis(mu):
        return -3 - mu

    def mask(self, parity):
        return self.even if parity == 0 else self.odd

    def fwd(self, f, mu, bc=1.0):
        """g(x) = f(x + mu-hat); the wrapped slab picks up ``bc`` when mu is time."""
        ax = self.axis(mu)
        g = torch.roll(f, shifts=-1, dims=ax)
        if mu == 3 and bc != 1.0:
            g = g.clone()
            idx = [slice(None)] * g.dim()
            idx[ax] = self.shape[0] - 1
            g[tuple(idx)] *= bc
        return g

    def bwd(self, f, mu, bc=1.0):
        """g(x) = f(x - mu-hat); the wrapped slab picks up ``bc`` when mu is time."""
        ax = self.axis(mu)
        g = torch.roll(f, shifts=1, dims=ax)
        if mu == 3 and bc != 1.0:
            g = g.clone()
            idx = [slice(None)] * g.dim()
            idx[ax] = 0
            g[tuple(idx)] *= bc
        return g

    # fermion shifts carry the time boundary factor
    def ffwd(self, psi, mu):
        return self.fwd(psi, mu, self.bc_t)

    def fbwd(self, psi, mu):
        return self.bwd(psi, mu, self.bc_t)

    def zeros_spinor(self, *batch):
        return torch.zeros(*batch, *self.shape, 4, 3, dtype=C128)

    def site_index(self):
        """Canonical lexicographic index x + Lx (y + Ly (z + Lz t)) of every site."""
        x, y, z, t = self.coords
        Lx, Ly, Lz, _ = self.dims
        return x + Lx * (y + Ly * (z + Lz * t))
