"""The library's scheme tables (host logic, no GPU) against the oracle's: both are written
from the action definitions of Sec. 2.2, 2.3, 2.5 and 3.6."""
import pytest

from test_gpu_multifilter import KIND, SCHEMES


@pytest.mark.parametrize("name", list(SCHEMES))
def test_scheme_term_lists(name):
    """The library's scheme tables equal the oracle's (both written from Sec. 2 and 3.6)."""
    from oracle.action import scheme
    from paper_1609_02652_gb300 import capi

    cid, p1, p2, kw = SCHEMES[name]
    d = capi.pfmp_action_scheme(cid, p1, p2, capi.ActionDef())
    ref = scheme(name, **kw)
    assert d.nterms == len(ref)
    for i, t in enumerate(ref):
        got = d.term[i]
        assert (got.kind, got.a, got.p1, got.p2) == (KIND[t.kind], t.a, t.p1, t.p2), (name, i)
        if t.kind == "ratio":
            assert got.b == t.b
