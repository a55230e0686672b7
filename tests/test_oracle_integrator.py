"""Pins of the oracle's integrators and trajectory: the paper's printed step arrays
(App. B), reversibility (App. B theorems) and the h^2 scaling of Delta H for 2MN."""
import json
import math
import os

import pytest
import torch

import pfmp_inputs as pin
from oracle.action import PFMP, PFMPParams
from oracle.integrator import LAMBDA_2MN, kinetic, leapfrog, link_update, merge, trajectory, two_mn
from oracle.lattice import Lattice, algebra_to_matrix, expi_hermitian

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _gold(h, lam):
    with open(os.path.join(GOLDEN, "integrator_arrays.json")) as f:
        g = json.load(f)

    def val(x):
        return x[0] * h + x[1] * lam * h

    return {k: {kk: [val(x) for x in vv] for kk, vv in v.items() if not kk.startswith("_")}
            for k, v in g.items() if not k.startswith("_")}


def test_printed_step_arrays():
    h, lam = 0.7, LAMBDA_2MN
    g = _gold(h, lam)
    T, S = leapfrog(2, h)
    assert T == pytest.approx(g["leapfrog_2step"]["T"], abs=1e-15)
    assert S == pytest.approx(g["leapfrog_2step"]["S"], abs=1e-15)
    T, S = leapfrog(3, h)
    assert T == pytest.approx(g["leapfrog_3step"]["T"]) and S == pytest.approx(g["leapfrog_3step"]["S"])
    T, S = two_mn(1, h)
    assert T == pytest.approx(g["2mn_1step"]["T"]) and S == pytest.approx(g["2mn_1step"]["S"])


def test_merge_worked_example():
    """3-step leapfrog + 1-step 2MN merge to the arrays of App. B 'Algorithm demonstration'."""
    h, lam = 1.0, LAMBDA_2MN
    g = _gold(h, lam)["merged_demo"]
    T, (S1, S2) = merge([leapfrog(3, h), two_mn(1, h)])
    assert T == pytest.approx(g["T"], abs=1e-14)
    assert S1 == pytest.approx(g["S1"], abs=1e-14)
    assert S2 == pytest.approx(g["S2"], abs=1e-14)


@pytest.mark.parametrize("steps", [(8, 16), (4, 10), (3, 5, 7)])
def test_merge_invariants(steps):
    """Sums of the merged arrays equal the trajectory length and the merged schedule is
    symmetric (Theorem: symmetric constituents give a reversible merged scheme)."""
    tau = 0.5
    T, Ss = merge([two_mn(n, tau) for n in steps])
    assert sum(T) == pytest.approx(tau, abs=1e-14)
    for S in Ss:
        assert sum(S) == pytest.approx(tau, abs=1e-14)
    # mirror: T'[1:] reversed equals T'[1:], S' reversed equals S'
    assert T[1:] == pytest.approx(T[1:][::-1], abs=1e-14)
    for S in Ss:
        assert S == pytest.approx(S[::-1], abs=1e-14)


def _cheap_setup(dims=(4, 4, 4, 4), n=4):
    lat = Lattice(dims, bc_t=-1)
    h = torch.tensor(pin.gauge_algebra(lat.dims, 1)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), 0.3)
    act = PFMP(lat, PFMPParams(beta=5.5, kappa=0.12, kappa_h=0.11, csw=1.0, n=n, tol=1e-13))
    xi = [torch.tensor(pin.spinor(lat.dims, 10 + i)).reshape(*lat.shape, 4, 3) * lat.even for i in range(3)]
    p0 = torch.tensor(pin.momenta(lat.dims, 5)).reshape(*lat.shape, 4, 8)
    return lat, U, act, xi, p0


def test_reversibility():
    """Forward, flip P, forward again returns to the start (App. B time reversibility)."""
    lat, U, act, xi, p0 = _cheap_setup()
    levels = [["polycorr", "hasen"], ["gauge", "det", "poly"]]
    sched = merge([two_mn(2, 0.1), two_mn(3, 0.1)])
    out = trajectory(act, U, p0, xi, 0.0, levels, sched)
    # second leg: same pseudofermions (heatbath at U0), reversed momenta, from U1
    phis = out["phi"]
    back = _run_md(act, out["U1"], -out["p1"], phis, levels, sched)
    Uback, pback = back
    assert (Uback - U).abs().max() < 1e-11
    assert (pback + p0).abs().max() < 1e-10


def _run_md(act, U, p, phis, levels, sched):
    T, Slev = sched
    forces = {
        "gauge": lambda V: act.F_gauge(V), "det": lambda V: act.F_det(V),
        "poly": lambda V: act.F_poly(V, phis[0]), "polycorr": lambda V: act.F_polycorr(V, phis[1]),
        "hasen": lambda V: act.F_hasen(V, phis[2]),
    }
    for i in range(len(T)):
        if T[i] != 0.0:
            U = link_update(U, p, T[i])
        for j, names in enumerate(levels):
            if Slev[j][i] != 0.0:
                for nme in names:
                    p = p - Slev[j][i] * forces[nme](U)
    return U, p


@pytest.mark.slow
def test_delta_h_scales_as_h_squared():
    """2MN is second order: halving every step size divides Delta H by about 4."""
    lat, U, act, xi, p0 = _cheap_setup(dims=(2, 2, 2, 4), n=4)
    levels = [["polycorr", "hasen"], ["gauge", "det", "poly"]]
    dh = []
    for nc in (4, 8):
        sched = merge([two_mn(nc, 0.2), two_mn(2 * nc, 0.2)])
        dh.append(abs(trajectory(act, U, p0, xi, 0.0, levels, sched)["dH"]))
    ratio = dh[0] / dh[1]
    assert 3.3 < ratio < 4.7, dh


def test_kinetic_normalisation():
    """sum tr P^2 with P = sum p_a T_a equals (1/2) sum p_a^2 (tr T_a T_b = delta_ab / 2)."""
    p = torch.tensor(pin.momenta((2, 2, 2, 2), 1)).reshape(2, 2, 2, 2, 4, 8)
    P = algebra_to_matrix(p)
    ref = torch.einsum("...ij,...ji->", P, P).real.item()
    assert kinetic(p) == pytest.approx(ref, rel=1e-13)
