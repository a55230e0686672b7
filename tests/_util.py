"""Helpers shared by the tests: oracle fields in canonical layout and device buffers for
the C-ABI.  The oracle side and the CUDA side only meet here, through the canonical
arrays (seeded inputs from pfmp_inputs)."""
import numpy as np
import torch

import pfmp_inputs as pin


def oracle_gauge(dims, eps, seed, bc_t=-1):
    from oracle.lattice import Lattice, algebra_to_matrix, expi_hermitian

    lat = Lattice(dims, bc_t=bc_t)
    h = torch.tensor(pin.gauge_algebra(dims, seed)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), eps)
    return lat, U


def canon(t):
    """Canonical float64 array of a complex oracle tensor (site-major, x fastest)."""
    return np.ascontiguousarray(torch.view_as_real(t.contiguous()).numpy()).reshape(-1)


def from_canon(a, lat, tail):
    return torch.view_as_complex(torch.tensor(np.asarray(a).reshape(*lat.shape, *tail, 2)))


def rel_l2(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


class Gpu:
    """A context on the GPU holding the same gauge field as the oracle."""

    def __init__(self, lat, U, stream=None):
        from paper_1609_02652_gb300 import capi

        self.capi = capi
        self.lat = lat
        self.ctx = capi.pfmp_ctx_create(lat.dims, lat.bc_t, stream)
        capi.pfmp_gauge_set(self.ctx, canon(U), capi.PFMP_HOST)
        self.ops = []

    def op(self, kappa, csw):
        o = self.capi.pfmp_op_create(self.ctx, kappa, csw)
        self.ops.append(o)
        return o

    def buf(self, prec):
        n = self.capi.pfmp_spinor_bytes(self.ctx, prec)
        dt = torch.float64 if prec == self.capi.PFMP_F64 else torch.float32
        return torch.zeros(n // dt.itemsize, dtype=dt, device="cuda")

    def pack(self, psi, prec, parity=0):
        b = self.buf(prec)
        self.capi.pfmp_spinor_pack(self.ctx, b, prec, canon(psi), self.capi.PFMP_HOST, parity)
        return b

    def unpack(self, b, prec, parity=0):
        out = np.zeros(self.lat.V * 24)
        self.capi.pfmp_spinor_unpack(self.ctx, out, self.capi.PFMP_HOST, b, prec, parity)
        return from_canon(out, self.lat, (4, 3))

    def close(self):
        for o in self.ops:
            self.capi.pfmp_op_destroy(o)
        self.ops = []
        self.capi.pfmp_ctx_destroy(self.ctx)
