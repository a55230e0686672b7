"""<exp(-dH)> = 1 for the oracle's PF-MP HMC (Sec. 2.1: the Metropolis step makes the
algorithm exact because the MD map is reversible and area-preserving; then the average
of exp(-dH) over the equilibrium distribution is exactly one).

The chain carries every PF-MP term of Sec. 2.5 (gauge, clover determinant, filter P_n(J),
filter correction [J P_n(J)]^{-1}, Hasenbusch ratio J K^{-1}) on a 2x2x2x4 lattice.  The
oracle is overhead-bound at this size (about five seconds per trajectory), so eight
independent chains run in spawned processes; each starts from a nearly Haar-random field
(U = exp(i 2.5 H)) at a weak coupling (beta = 0.5), which is close to the equilibrium
distribution from the start.  A wrong Hamiltonian (kinetic normalisation, a term's
action evaluated with another pseudofermion than its heatbath drew, a term missing from
H but present in the MD) or an MD map that is not reversible moves the mean by far more
than the statistical bar.
"""
import math
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

DIMS = (2, 2, 2, 4)
N_CHAINS = 8
N_TRAJ = 22
N_SKIP = 2


def _chain(seed):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    torch.set_num_threads(1)
    import pfmp_inputs as pin
    from oracle.action import PFMP, PFMPParams
    from oracle.integrator import merge, trajectory, two_mn
    from oracle.lattice import Lattice, algebra_to_matrix, expi_hermitian

    lat = Lattice(DIMS, bc_t=-1)
    h = torch.tensor(pin.gauge_algebra(DIMS, 500 + seed)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), 2.5)
    act = PFMP(lat, PFMPParams(beta=0.5, kappa=0.11, kappa_h=0.10, csw=1.0, n=4, tol=1e-11))
    sched = merge([two_mn(1, 0.5)])
    levels = [["gauge", "det", "poly", "polycorr", "hasen"]]
    out = []
    for k in range(N_TRAJ):
        s = 10000 * (seed + 1) + k
        p0 = torch.tensor(pin.momenta(DIMS, s)).reshape(*lat.shape, 4, 8)
        xi = [lat.even * torch.tensor(pin.spinor(DIMS, 3 * s + j)).reshape(*lat.shape, 4, 3) for j in range(3)]
        r = trajectory(act, U, p0, xi, float(pin.uniform(s)[0]), levels, sched)
        U = r["U"]
        out.append((r["dH"], r["accepted"]))
    return out


@pytest.mark.slow
def test_exp_minus_delta_h_is_one_with_fermion_terms():
    workers = min(N_CHAINS, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(workers) as pool:
        chains = pool.map(_chain, range(N_CHAINS))
    dH = np.array([d for c in chains for d, _ in c[N_SKIP:]])
    acc = np.array([a for c in chains for _, a in c[N_SKIP:]])
    ex = np.exp(-dH)
    # the chains are independent; within a chain exp(-dH) is close to uncorrelated
    # (momenta and noise are redrawn every trajectory): tau_int taken as 2
    err = math.sqrt(2 * 2.0) * ex.std(ddof=1) / math.sqrt(len(ex))
    assert dH.std() > 1e-2, dH.std()                 # the test is not trivially satisfied
    assert abs(ex.mean() - 1.0) < 4 * err, (ex.mean(), err)
    assert acc.mean() > 0.5
