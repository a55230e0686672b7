"""Writes cg_iterations_16x16x16x32.json: the number of FP64 CG iterations the ORACLE needs
to bring the 16^3x32 benchmark system (eps=0.5 random SU(3), c_sw=1.0, kappa=0.130,
Gaussian RHS seed 100, zero initial guess) to a true relative residual below 1e-10, and
the oracle's residual history.  Calls only oracle/ and pfmp_inputs.

    python tests/golden/make_cg_iterations.py
"""
import json
import math
import os
import sys
import time

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import pfmp_inputs as pin  # noqa: E402
from oracle.dirac import WilsonClover  # noqa: E402
from oracle.lattice import Lattice, algebra_to_matrix, expi_hermitian  # noqa: E402

DIMS, EPS, KAPPA, CSW, TOL = (16, 16, 16, 32), 0.5, 0.130, 1.0, 1e-10


def main():
    lat = Lattice(DIMS, bc_t=-1)
    h = torch.tensor(pin.gauge_algebra(DIMS, 1)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), EPS)
    W = WilsonClover(lat, U, KAPPA, CSW)
    b = torch.tensor(pin.spinor(DIMS, 100)).reshape(*lat.shape, 4, 3) * lat.even
    x = torch.zeros_like(b)
    r = b.clone()
    p = r.clone()
    rr = (r.conj() * r).sum().real
    bb = rr
    hist = []
    t0 = time.time()
    it = 0
    while math.sqrt(rr / bb) >= 0.5 * TOL and it < 5000:
        Ap = W.K(p)
        a = rr / (p.conj() * Ap).sum().real
        x = x + a * p
        r = r - a * Ap
        rn = (r.conj() * r).sum().real
        p = r + (rn / rr) * p
        rr = rn
        it += 1
        hist.append(math.sqrt(rr / bb))
        if it % 50 == 0:
            print(it, hist[-1], time.time() - t0, flush=True)
    res = float(torch.linalg.vector_norm(b - W.K(x)) / torch.linalg.vector_norm(b))
    out = {"_source": "oracle FP64 CG, written by tests/golden/make_cg_iterations.py",
           "dims": DIMS, "eps": EPS, "kappa": KAPPA, "csw": CSW, "tol": TOL, "iterations": it,
           "true_rel_res": res, "residual_history_every_10": hist[::10]}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "cg_iterations_16x16x16x32.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out["iterations"], res)


if __name__ == "__main__":
    main()
