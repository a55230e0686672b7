"""The allocation-free M-hat entry point (pfmp_mhat_noalloc).

Callers that may not allocate or free device memory while they run (a host callback or
a latency-bound loop with no room for an allocation, a framework whose memory pool owns
all device memory) use this variant; its odd-site temporary is a fixed array inside the
library instead of the operator's own buffer.  It runs the same kernels as pfmp_mhat, so
its output must be bit-identical, call after call (the array keeps the previous call's
contents); it must reject lattices whose temporary does not fit and the FP16-storage
precision.  This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import pytest
import torch

import pfmp_inputs as pin
from _util import Gpu, oracle_gauge

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
def test_mhat_noalloc_matches_mhat_twice(prec):
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge((6, 4, 4, 8), 0.4, 31)
    g = Gpu(lat, U)
    try:
        op = g.op(0.125, 1.0)
        for call, seed in enumerate((41, 42)):      # two calls in a row, different inputs
            psi = lat.even * torch.tensor(pin.spinor(lat.dims, seed)).reshape(*lat.shape, 4, 3)
            b_in = g.pack(psi, prec, 0)
            for dagger in (0, 1):
                ref = g.buf(prec)
                got = g.buf(prec)
                capi.pfmp_mhat(op, prec, ref, b_in, dagger)
                capi.pfmp_mhat_noalloc(op, prec, got, b_in, dagger)
                torch.cuda.synchronize()
                assert torch.equal(got, ref), (call, dagger)   # same kernels: bit-identical
                r = lat.even * g.unpack(ref, prec, 0)
                assert float(torch.linalg.vector_norm(r)) > 0
    finally:
        g.close()


def test_mhat_noalloc_rejects_oversized_lattice():
    from paper_1609_02652_gb300 import capi

    # FP64 temporary of 32^3 x 64 (1,048,576 sites per parity, 201 MB) exceeds 64 MiB
    ctx = capi.pfmp_ctx_create((32, 32, 32, 64), -1, None)
    try:
        import numpy as np

        h = np.zeros(32 * 32 * 32 * 64 * 32)
        capi.pfmp_gauge_from_algebra(ctx, h, 0.0, capi.PFMP_HOST)
        op = capi.pfmp_op_create(ctx, 0.12, 0.0)
        try:
            n = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F64) // 8
            a = torch.zeros(n, dtype=torch.float64, device="cuda")
            b = torch.zeros_like(a)
            with pytest.raises(capi.PfmpError) as e:
                capi.pfmp_mhat_noalloc(op, capi.PFMP_F64, b, a, 0)
            assert e.value.status == capi.PFMP_E_INVALID
            assert "exceeds the fixed scratch" in str(e.value)
        finally:
            capi.pfmp_op_destroy(op)
    finally:
        capi.pfmp_ctx_destroy(ctx)


def test_mhat_noalloc_rejects_fp16_storage():
    from paper_1609_02652_gb300 import capi

    lat, U = oracle_gauge((4, 4, 4, 8), 0.3, 5)
    g = Gpu(lat, U)
    try:
        op = g.op(0.12, 1.0)
        nb = capi.pfmp_spinor_bytes(g.ctx, capi.PFMP_H16)
        a = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        b = torch.zeros_like(a)
        with pytest.raises(capi.PfmpError) as e:
            capi.pfmp_mhat_noalloc(op, capi.PFMP_H16, b, a, 0)
        assert e.value.status == capi.PFMP_E_INVALID
        assert "PFMP_F64 or PFMP_F32" in str(e.value)
    finally:
        g.close()
