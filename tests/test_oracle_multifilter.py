"""Pins of the oracle's general filtered / mass-preconditioned actions (Sec. 2.2, 2.3,
2.5, 3.6; App. A factorisation; App. C forces): the factorised filter Q = P_p2 / P_p1,
each term's action against a dense operator assembled from its definition, the
determinant identity of every scheme (the product of the term determinants is det K),
the heatbath identities, and the new force forms against finite differences."""
import pytest
import torch

import pfmp_inputs as pin
from oracle import cheby
from oracle.action import Action, Term, scheme
from oracle.dirac import WilsonClover, dense, from_parity_vector, to_parity_vector
from oracle.lattice import C128, F64, Lattice, algebra_to_matrix, expi_hermitian

MU, NU = 1.2, 0.9


@pytest.mark.parametrize("p1,p2", [(4, 24), (4, 14), (2, 8), (6, 48), (8, 26), (12, 64), (12, 38)])
def test_filter_factorisation(p1, p2):
    """P_p1(z) Q(z) = P_p2(z) at arbitrary complex z, with q = p2 - p1 roots."""
    z, c = cheby.filter_roots(p1, p2, MU, NU)
    assert z.numel() == p2 - p1
    x = torch.tensor([0.3 + 0.2j, 1.7 - 0.4j, -0.5 + 1.1j, 2.2 + 0.0j], dtype=C128)
    q = c * torch.prod(x[:, None] - z, -1)
    lhs = cheby.poly_scalar(x, p1, MU, NU) * q
    rhs = cheby.poly_scalar(x, p2, MU, NU)
    assert ((lhs - rhs).abs() / rhs.abs()).max() < 1e-12
    # Q is positive on the real axis and its roots close under conjugation
    xr = torch.linspace(0.05, 2.5, 50, dtype=F64).to(C128)
    qr = c * torch.prod(xr[:, None] - z, -1)
    assert (qr.imag.abs() < 1e-12 * qr.abs()).all() and (qr.real > 0).all()
    assert torch.allclose(torch.sort(z.conj().real)[0], torch.sort(z.real)[0])


def test_filter_orders_rejected():
    with pytest.raises(ValueError):
        cheby.filter_roots(12, 48, MU, NU)     # 13 does not divide 49
    with pytest.raises(ValueError):
        cheby.filter_roots(4, 4, MU, NU)
    with pytest.raises(ValueError):
        cheby.filter_roots(0, 7, MU, NU)
    z, c = cheby.filter_roots(0, 8, MU, NU)
    assert torch.equal(z, cheby.roots(8, MU, NU)) and c == cheby.norm(8, MU, NU)


@pytest.fixture(scope="module")
def tiny():
    lat = Lattice((2, 2, 2, 2), bc_t=-1)
    h = torch.tensor(pin.gauge_algebra(lat.dims, 4)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), 0.5)
    kappas = [0.125, 0.105, 0.115]
    D = {}
    for a, k in enumerate(kappas):
        W = WilsonClover(lat, U, k, 1.2)
        D[a] = (dense(lat, W.mhat), dense(lat, W.K))
    return lat, U, kappas, D


def _dense_term(t, D, kappas):
    """The term's operator O (S = phi^dag O phi) assembled from its definition."""
    Wa, Ja = D[t.a]
    I = torch.eye(Ja.shape[0], dtype=C128)
    if t.kind == "filter":
        # Q = P_p2 / P_p1 from the two dense polynomials (P_0 = 1)
        def P(p):
            X = cheby.norm(p, MU, NU) * I
            for z in cheby.roots(p, MU, NU):
                X = X @ (Ja - z * I)
            return X
        return torch.linalg.solve(P(t.p1), P(t.p2)) if t.p1 else P(t.p2)
    if t.kind == "filtercorr":
        X = cheby.norm(t.p2, MU, NU) * Ja
        for z in cheby.roots(t.p2, MU, NU):
            X = X @ (Ja - z * I)
        return torch.linalg.inv(X)
    if t.kind == "ratio":
        return Wa @ torch.linalg.solve(D[t.b][1], Wa.conj().T)
    return torch.linalg.inv(Ja)


@pytest.mark.parametrize("name,kw", [("1PF", dict(p2=8)), ("2PF", dict(p1=4, p2=14)), ("1MP", {}), ("2MP", {}),
                                     ("PF-MP", dict(p2=8)), ("2PF-1MP", dict(p1=4, p2=24)),
                                     ("1PF-2MP", dict(p2=4))])
def test_scheme_terms_and_determinant(tiny, name, kw):
    """Each fermion term's S(phi) equals phi^dag O phi with O assembled densely, and
    prod_i det O_i^{-1} = det K (every scheme samples the same two-flavour determinant)."""
    lat, U, kappas, D = tiny
    act = Action(lat, 5.5, 1.2, kappas, scheme(name, **kw), mu=MU, nu=NU, tol=1e-13)
    ld = lambda X: torch.linalg.slogdet(X)[1].item()
    total = 0.0
    for k, i in enumerate(act.pf):
        t = act.terms[i]
        O = _dense_term(t, D, kappas)
        assert (O - O.conj().T).abs().max() < 1e-9 * O.abs().max()
        total -= ld(O)
        phi = lat.even * torch.tensor(pin.spinor(lat.dims, 40 + k)).reshape(*lat.shape, 4, 3)
        v = to_parity_vector(lat, phi)
        ref = (v.conj() @ O @ v).real.item()
        assert abs(act.S(U, i, phi).item() - ref) < 1e-9 * abs(ref), (name, t)
    assert abs(total - ld(D[0][1])) < 1e-8, name


@pytest.fixture(scope="module")
def small():
    lat = Lattice((4, 4, 4, 4), bc_t=-1)
    h = torch.tensor(pin.gauge_algebra(lat.dims, 1)).reshape(*lat.shape, 4, 8)
    U = expi_hermitian(algebra_to_matrix(h), 0.3)
    return lat, U


@pytest.mark.parametrize("name,kw,kappas", [("2PF-1MP", dict(p1=2, p2=8), [0.12, 0.11]),
                                            ("1PF-2MP", dict(p2=4), [0.12, 0.10, 0.11]),
                                            ("2MP", {}, [0.12, 0.10, 0.11])])
def test_heatbath_identity(small, name, kw, kappas):
    lat, U = small
    act = Action(lat, 5.5, 1.0, kappas, scheme(name, **kw))
    xi = [lat.even * torch.tensor(pin.spinor(lat.dims, 20 + k)).reshape(*lat.shape, 4, 3) for k in range(len(act.pf))]
    phis = act.heatbath(U, xi)
    for k, i in enumerate(act.pf):
        ref = (xi[k].abs() ** 2).sum().item()
        assert abs(act.S(U, i, phis[k]).item() - ref) < 1e-10 * ref


def _fd(S, U, site, mu, a, d=1e-4):
    def f(e):
        V = U.clone()
        h = torch.zeros(8, dtype=F64)
        h[a] = e
        V[site][mu] = expi_hermitian(algebra_to_matrix(h), 1.0) @ U[site][mu]
        return float(S(V))
    return (8 * (f(d) - f(-d)) - (f(2 * d) - f(-2 * d))) / (12 * d)


LINKS = [((1, 2, 3, 0), 2, 5), ((3, 1, 0, 2), 0, 7), ((2, 3, 1, 1), 1, 2)]


@pytest.mark.parametrize("term", [Term("filter", a=1, p1=2, p2=8), Term("filter", a=0, p1=4, p2=14),
                                  Term("inv", a=1), Term("ratio", a=1, b=2)],
                         ids=["Q(J)", "Q(K)", "inv", "ratio"])
def test_force_against_finite_difference(small, term):
    lat, U = small
    act = Action(lat, 5.5, 1.0, [0.12, 0.10, 0.11], [term])
    phi = lat.even * torch.tensor(pin.spinor(lat.dims, 31)).reshape(*lat.shape, 4, 3)
    F = act.F(U, 0, phi)
    scale = F.abs().max().item()
    for site, mu, a in LINKS:
        fd = _fd(lambda V: act.S(V, 0, phi), U, site, mu, a)
        assert abs(F[site][mu][a].item() - fd) < 1e-7 * scale, (term, site, mu, a)


def test_ratio_degenerate_limit(small):
    """a = b: W_a K_a^{-1} W_a^dag = 1, S = phi^dag phi, zero force."""
    lat, U = small
    act = Action(lat, 5.5, 1.0, [0.12, 0.11], [Term("ratio", a=1, b=1)])
    phi = lat.even * torch.tensor(pin.spinor(lat.dims, 3)).reshape(*lat.shape, 4, 3)
    s = act.S(U, 0, phi).item()
    assert abs(s - (phi.abs() ** 2).sum().item()) < 1e-10 * s
    assert act.F(U, 0, phi).abs().max() < 1e-9
